// Near field (List 1, step 3 of Sec. 6.4) and the direct sum (Sec. 2.3,
// Eq. evaluation_problem) for 2D/3D Laplace and Helmholtz, single and double
// layer, in float64 / complex128.
//
// Layout: one CTA per target leaf. 128 threads = 32 targets x 4 source
// lanes; the sources of each List-1 leaf are staged through shared memory
// in chunks; the 4 partial sums of a target are combined in a fixed order,
// so results are bitwise reproducible.
#include "cfmm_special.cuh"
#include "kernels.cuh"

namespace cfmm {

void upload_lag_rule_p2p() { upload_lag_rule_local(); }

constexpr int kP2PThreads = 128;
constexpr int kP2PTargets = 32;
constexpr int kP2PSplit = kP2PThreads / kP2PTargets;
constexpr int kP2PChunk = 128;

// K(x, y) sigma + (n . grad_y K)(x, y) tau for one pair (d = x - y != 0)
template <int DIM, int KER>
__device__ __forceinline__ void pair_kernel(const double* dr, const double* di, const double* nr,
                                            const double* ni, cd sg, cd ta, bool slp, bool dlp,
                                            double kappa, cd& acc) {
    cd d[DIM];
    cd r2 = {0.0, 0.0};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        d[a] = cd{dr[a], di[a]};
        r2 += d[a] * d[a];
    }
    cd nd = {0.0, 0.0};
    if (dlp) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) nd += cd{nr[a], ni[a]} * d[a];
    }
    if (DIM == 2 && KER == CFMM_LAPLACE) {
        // log r = Log(r^2)/2 ; grad_y log r = (y - x)/r^2
        if (slp) acc += (0.5 * clog_p(r2)) * sg;
        if (dlp) acc -= (nd / r2) * ta;
    } else if (DIM == 2) {
        cd r = csqrt_p(r2);
        cd h0, h1;
        hankel01(kappa * r, &h0, &h1);
        if (slp) acc += h0 * sg;
        if (dlp) acc += (kappa * h1) * (nd / r) * ta;
    } else if (KER == CFMM_LAPLACE) {
        cd r = csqrt_p(r2);
        cd ir = cinv(r);
        if (slp) acc += ir * sg;
        if (dlp) acc += (nd * (ir * ir * ir)) * ta;
    } else {
        cd r = csqrt_p(r2);
        cd ir = cinv(r);
        cd e = cexp_i(kappa * r);
        cd g = e * ir;
        if (slp) acc += g * sg;
        if (dlp) acc += (nd * (cd{1.0, 0.0} - mul_i(kappa * r)) * g * (ir * ir)) * ta;
    }
}

struct SrcTile {
    double re[kP2PChunk][3];
    double im[kP2PChunk][3];
    double nr[kP2PChunk][3];
    double ni[kP2PChunk][3];
    cd sg[kP2PChunk];
    cd ta[kP2PChunk];
};

template <int DIM, int KER>
__device__ void accumulate_sources(SrcTile& S, const KParams& K, int rhs, int s, int e, int ti, bool tvalid,
                                   const double* xr, const double* xim, cd& acc, int split) {
    const int64_t n = K.n_src;
    for (int c0 = s; c0 < e; c0 += kP2PChunk) {
        int cn = min(kP2PChunk, e - c0);
        __syncthreads();
        for (int j = threadIdx.x; j < cn; j += blockDim.x) {
            int g = c0 + j;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                S.re[j][a] = K.src_re[a * n + g];
                S.im[j][a] = K.src_im[a * n + g];
                if (K.dlp) {
                    S.nr[j][a] = K.nrm_re[a * n + g];
                    S.ni[j][a] = K.nrm_im[a * n + g];
                }
            }
            if (K.slp) S.sg[j] = K.sigma[(int64_t)rhs * K.dens_stride + g];
            if (K.dlp) S.ta[j] = K.tau[(int64_t)rhs * K.dens_stride + g];
        }
        __syncthreads();
        if (tvalid) {
            for (int j = split; j < cn; j += kP2PSplit) {
                double dr[DIM], di[DIM];
                bool zero = true;
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    dr[a] = xr[a] - S.re[j][a];
                    di[a] = xim[a] - S.im[j][a];
                    zero = zero && dr[a] == 0.0 && di[a] == 0.0;
                }
                if (zero) continue;   // x == y: self pair / coincident point
                pair_kernel<DIM, KER>(dr, di, S.nr[j], S.ni[j], K.slp ? S.sg[j] : cd{0, 0},
                                      K.dlp ? S.ta[j] : cd{0, 0}, K.slp, K.dlp, K.kappa, acc);
            }
        }
    }
}

template <int DIM, int KER>
__device__ void finish_target(cd acc, cd* red, int tl, int split, bool tvalid, cd* out, bool add) {
    red[split * kP2PTargets + tl] = acc;
    __syncthreads();
    if (split == 0 && tvalid) {
        cd s = red[tl];
        for (int q = 1; q < kP2PSplit; ++q) s += red[q * kP2PTargets + tl];
        if (add) *out += s;
        else *out = s;
    }
    __syncthreads();
}

// near field over List 1; out = sorted potential [rhs][n] (overwritten)
template <int DIM, int KER>
__global__ void __launch_bounds__(kP2PThreads) k_p2p(KParams K, const int* __restrict__ leaf_boxes,
                                                     const int* __restrict__ bst, const int* __restrict__ ben,
                                                     const int* __restrict__ l1off, const int* __restrict__ l1,
                                                     cd* __restrict__ out, int add) {
    __shared__ SrcTile S;
    __shared__ cd red[kP2PThreads];
    int b = leaf_boxes[blockIdx.x];
    int rhs = blockIdx.y;
    int tl = threadIdx.x % kP2PTargets, split = threadIdx.x / kP2PTargets;
    int ts = bst[b], te = ben[b];
    for (int t0 = ts; t0 < te; t0 += kP2PTargets) {
        int ti = t0 + tl;
        bool tvalid = ti < te;
        double xr[DIM], xim[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            xr[a] = tvalid ? K.trg_re[a * K.n_trg + ti] : 0.0;
            xim[a] = tvalid ? K.trg_im[a * K.n_trg + ti] : 0.0;
        }
        cd acc = {0.0, 0.0};
        for (int q = l1off[b]; q < l1off[b + 1]; ++q) {
            int a = l1[q];
            accumulate_sources<DIM, KER>(S, K, rhs, bst[a], ben[a], ti, tvalid, xr, xim, acc, split);
        }
        finish_target<DIM, KER>(acc, red, tl, split, tvalid, out + (int64_t)rhs * K.n_trg + ti, add != 0);
    }
}

// direct sum: every target against every source
template <int DIM, int KER>
__global__ void __launch_bounds__(kP2PThreads) k_direct(KParams K, cd* __restrict__ out) {
    __shared__ SrcTile S;
    __shared__ cd red[kP2PThreads];
    int rhs = blockIdx.y;
    int tl = threadIdx.x % kP2PTargets, split = threadIdx.x / kP2PTargets;
    int ti = blockIdx.x * kP2PTargets + tl;
    bool tvalid = ti < K.n_trg;
    double xr[DIM], xim[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        xr[a] = tvalid ? K.trg_re[a * K.n_trg + ti] : 0.0;
        xim[a] = tvalid ? K.trg_im[a * K.n_trg + ti] : 0.0;
    }
    cd acc = {0.0, 0.0};
    accumulate_sources<DIM, KER>(S, K, rhs, 0, (int)K.n_src, ti, tvalid, xr, xim, acc, split);
    finish_target<DIM, KER>(acc, red, tl, split, tvalid, out + (int64_t)rhs * K.n_trg + ti, false);
}

template <int DIM, int KER>
static void launch_p2p_t(const KParams& K, const int* leaf_boxes, int nleaves, const int* bst, const int* ben,
                         const int* l1off, const int* l1, cd* out, int nrhs, bool add, cudaStream_t st) {
    if (nleaves == 0) return;
    dim3 grid(nleaves, nrhs);
    k_p2p<DIM, KER><<<grid, kP2PThreads, 0, st>>>(K, leaf_boxes, bst, ben, l1off, l1, out, add ? 1 : 0);
    CFMM_LAUNCHED();
}

void launch_p2p(int dim, int ker, const KParams& K, const int* leaf_boxes, int nleaves, const int* bst,
                const int* ben, const int* l1off, const int* l1, cd* out, int nrhs, bool add, cudaStream_t st) {
    if (dim == 2 && ker == CFMM_LAPLACE) launch_p2p_t<2, CFMM_LAPLACE>(K, leaf_boxes, nleaves, bst, ben, l1off, l1, out, nrhs, add, st);
    else if (dim == 2) launch_p2p_t<2, CFMM_HELMHOLTZ>(K, leaf_boxes, nleaves, bst, ben, l1off, l1, out, nrhs, add, st);
    else if (ker == CFMM_LAPLACE) launch_p2p_t<3, CFMM_LAPLACE>(K, leaf_boxes, nleaves, bst, ben, l1off, l1, out, nrhs, add, st);
    else launch_p2p_t<3, CFMM_HELMHOLTZ>(K, leaf_boxes, nleaves, bst, ben, l1off, l1, out, nrhs, add, st);
}

template <int DIM, int KER>
static void launch_direct_t(const KParams& K, cd* out, int nrhs, cudaStream_t st) {
    dim3 grid((unsigned)((K.n_trg + kP2PTargets - 1) / kP2PTargets), nrhs);
    k_direct<DIM, KER><<<grid, kP2PThreads, 0, st>>>(K, out);
    CFMM_LAUNCHED();
}

void launch_direct(int dim, int ker, const KParams& K, cd* out, int nrhs, cudaStream_t st) {
    if (K.n_trg == 0) return;
    if (dim == 2 && ker == CFMM_LAPLACE) launch_direct_t<2, CFMM_LAPLACE>(K, out, nrhs, st);
    else if (dim == 2) launch_direct_t<2, CFMM_HELMHOLTZ>(K, out, nrhs, st);
    else if (ker == CFMM_LAPLACE) launch_direct_t<3, CFMM_LAPLACE>(K, out, nrhs, st);
    else launch_direct_t<3, CFMM_HELMHOLTZ>(K, out, nrhs, st);
}

}  // namespace cfmm
