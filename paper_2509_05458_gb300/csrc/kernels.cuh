// Launch interfaces of the apply-path kernels (shared by the .cu files).
#pragma once

#include "cfmm_common.cuh"

namespace cfmm {

// Geometry and densities seen by the point-wise kernels. Points are SoA
// [dim][n] float64 (sorted order); densities are complex128 with a stride of
// dens_stride between right-hand sides.
struct KParams {
    const double* src_re;
    const double* src_im;
    const double* nrm_re;
    const double* nrm_im;
    const double* trg_re;
    const double* trg_im;
    int64_t n_src, n_trg;
    const cd* sigma;
    const cd* tau;
    int64_t dens_stride;
    bool slp, dlp;
    double kappa;
};

// near field of an apply on the plan's side stream: near_fork() makes the
// side stream wait for what the plan's stream has queued and returns it;
// near_join() makes the plan's stream wait for the side stream. In the
// serialised timing mode near_fork() returns the plan's stream itself and
// near_launched(), called right after the near-field launch, closes its
// timing bracket.
cudaStream_t near_fork(cfmm_plan_s* P);
void near_launched(cfmm_plan_s* P);
void near_join(cfmm_plan_s* P);
// blevel/W/sep: the tree's box levels, root width and separation (the mixed
// 3D Helmholtz near field sizes its coordinate grid from them; NULL = unknown)
void launch_p2p(int dim, int ker, const KParams& K, const int* leaf_boxes, int nleaves, const int* bst,
                const int* ben, const int* l1off, const int* l1, cd* out, int nrhs, bool add, cudaStream_t st,
                bool mixed = false, const int* blevel = nullptr, double W = 0.0, int sep = 1);
void launch_direct(int dim, int ker, const KParams& K, cd* out, int nrhs, cudaStream_t st, bool mixed = false);
// near-field target gradient over List 1 in FP64: g = sorted [nrhs][dim][n], overwritten
void launch_p2p_grad(int dim, int ker, const KParams& K, const int* leaf_boxes, int nleaves, const int* bst,
                     const int* ben, const int* l1off, const int* l1, cd* g, int nrhs, cudaStream_t st);

// tree construction (tree.cu)
void build_tree(cfmm_plan_s* P, const double* re, const double* im, const double* nre, const double* nim,
                int top_level_opt);
// Lists 1-4 of the plan's tree (after build_tree)
void build_plan_lists(cfmm_plan_s* P);

// 2D expansions (fmm2d.cu)
// 2D expansions: fmm2d_presetup before the lists (orders, leaves, the per-point
// row table on the side stream), fmm2d_setup after them
void fmm2d_presetup(cfmm_plan_s* P);
void fmm2d_setup(cfmm_plan_s* P);
void fmm2d_release(cfmm_plan_s* P);
// g: sorted target gradient [nrhs][dim][n] (overwritten) or NULL
void fmm2d_apply(cfmm_plan_s* P, const cd* sigma, const cd* tau, int64_t dens_stride, cd* out_sorted, int nrhs,
                 cd* g = nullptr);

// Green's function constants of CFMM_GREEN_SCALE: -1/(2 pi) (2D Laplace),
// i/4 (2D Helmholtz), 1/(4 pi) (3D Laplace and Helmholtz)
inline cd green_scale(int dim, int ker) {
    const double pi = 3.14159265358979323846;
    if (dim == 2 && ker == CFMM_LAPLACE) return cd{-1.0 / (2.0 * pi), 0.0};
    if (dim == 2) return cd{0.0, 0.25};
    return cd{1.0 / (4.0 * pi), 0.0};
}
// true for device (or managed) memory (api.cu); a CUDA call
bool is_device_ptr(const void* p);
// v[i] *= s for i < cnt (direct_noalloc.cu)
void launch_scale_inplace(cd* v, int64_t cnt, cd s, cudaStream_t st);

// direct sum with library-owned fixed scratch (direct_noalloc.cu); validates
// every argument it can without a CUDA call before touching the GPU
int direct_noalloc(int dim, int kernel, double k, const double* src_re, const double* src_im, const double* nrm_re,
                   const double* nrm_im, int64_t m, const double* trg_re, const double* trg_im, int64_t n,
                   const double* densities, int nrhs, double* out, void* stream);

// 3D Laplace expansions (fmm3d.cu)
void fmm3d_setup(cfmm_plan_s* P);
void fmm3d_release(cfmm_plan_s* P);
// g: sorted target gradient [nrhs][dim][n] (overwritten) or NULL
void fmm3d_apply(cfmm_plan_s* P, const cd* sigma, const cd* tau, int64_t dens_stride, cd* out_sorted, int nrhs,
                 cd* g = nullptr);

// 3D Helmholtz expansions (helm3d.cu)
void helm3d_setup(cfmm_plan_s* P);
void helm3d_release(cfmm_plan_s* P);
// g: sorted target gradient [nrhs][dim][n] (overwritten) or NULL
void helm3d_apply(cfmm_plan_s* P, const cd* sigma, const cd* tau, int64_t dens_stride, cd* out_sorted, int nrhs,
                 cd* g = nullptr);
int nterms_helm3d(int k, double eps, double kappa, double w);
// 3D Laplace point-and-shoot translations (helm3d.cu, used by fmm3d.cu)
// largest 3D Helmholtz expansion order: the limit of the translation tables
// (the translation kernel keeps 3 (P+1)^2 + 10 P + 5 complex values in shared
// memory, the rest in global scratch, which fits up to here)
constexpr int kMaxP3Top = 63;
struct Lap3Tr;
Lap3Tr* lap3_tr_create(cfmm_plan_s* P, int Pord);
void lap3_tr_destroy(Lap3Tr* L);
// single-layer 3D Laplace P2M over `leaves` (one column per lane); false when
// the order does not fit the kernel (the caller then uses the general P2M)
bool lap3_p2m_slp(Lap3Tr* L, cfmm_plan_s* P, const int* leaves, int cnt, int maxP, const int* dPlev,
                  const int64_t* eoff, int64_t ncoef, const cd* sigma, int64_t dstride, cd* out, int nrhs);
void lap3_tr_launch(Lap3Tr* L, cfmm_plan_s* P, int mode, int l, int Pord, const int64_t* eoff, int64_t ncoef,
                    const cd* in, cd* out, int nrhs);
// single-layer 3D Laplace P2M with complex64 products and FP64 sums over
// `leaves` (writes their multipoles); false when the order does not fit
bool lap3_p2m32(Lap3Tr* L, cfmm_plan_s* P, const int* leaves, int cnt, int maxP, const int* dPlev,
                const int64_t* eoff, int64_t ncoef, const cd* sigma, int64_t dstride, cd* out, int nrhs);
// 3D Laplace L2P in complex64 arithmetic over `leaves` (adds to u)
void lap3_l2p32(Lap3Tr* L, cfmm_plan_s* P, const int* leaves, int cnt, int maxP, const int* dPlev,
                const int64_t* eoff, int64_t ncoef, const cd* loc, cd* u, int nrhs);

void upload_lag_rule_p2p();
void upload_lag_rule_fmm2d();

}  // namespace cfmm
