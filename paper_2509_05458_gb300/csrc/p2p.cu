// Near field (List 1, step 3 of Sec. 6.4) and the direct sum (Sec. 2.3,
// Eq. evaluation_problem) for 2D/3D Laplace and Helmholtz, single and double
// layer, in float64 / complex128 or in mixed precision (complex64 kernel
// arithmetic, FP32 hi/lo pair differences, compensated sums).
//
// Layout: one CTA per target leaf. 128 threads = 32 targets x 4 source
// lanes; the sources of each List-1 leaf are staged through shared memory
// in chunks; the 4 partial sums of a target are combined in a fixed order,
// so results are bitwise reproducible.
#include "cfmm_special.cuh"
#include "kernels.cuh"

namespace cfmm {

// ---------------------------------------------------------------------------
// Ascending series of H_0^(1), H_1^(1) in w = -(kappa r)^2/4 (DLMF 10.2.2,
// 10.8.1), evaluated by Horner's rule with precomputed coefficients:
//   A(w) = sum w^k/(k!)^2                   J_0 = A
//   B(w) = sum w^k/(k!(k+1)!)               J_1 = (z/2) B
//   C(w) = sum_{k>=1} H_k w^k/(k!)^2        Y_0 = (2/pi)((log(z/2)+gamma) A - C)
//   D(w) = sum (psi(k+1)+psi(k+2)) w^k/(k!(k+1)!)
//                                           Y_1 = -2/(pi z) + (2/pi) log(z/2) J_1 - (z/(2pi)) D
// with H_k the harmonic numbers and psi(k+1) = -gamma + H_k. Only r^2 enters:
// log(z/2) = Log(q)/2 with q = (kappa r/2)^2, and the double layer needs
// kappa J_1/r = (kappa^2/2) B and kappa Y_1/r = -2/(pi r^2) + (kappa^2/pi) log(z/2) B
// - (kappa^2/(2 pi)) D, so the near field takes no square root.
// ---------------------------------------------------------------------------
constexpr int kSerMax = 21;
struct SeriesTab {
    double a[kSerMax + 1], b[kSerMax + 1], c[kSerMax + 1], d[kSerMax + 1];
    float af[kSerMax + 1], bf[kSerMax + 1], cf_[kSerMax + 1], df[kSerMax + 1];
};
static __constant__ SeriesTab c_ser;

static SeriesTab make_series_tab() {
    SeriesTab T;
    const double g = 0.57721566490153286061;
    double fk = 1.0, H = 0.0;   // k!, H_k
    for (int k = 0; k <= kSerMax; ++k) {
        if (k > 0) {
            fk *= k;
            H += 1.0 / k;
        }
        double fk1 = fk * (k + 1);
        T.a[k] = 1.0 / (fk * fk);
        T.b[k] = 1.0 / (fk * fk1);
        T.c[k] = H / (fk * fk);
        T.d[k] = (-2.0 * g + 2.0 * H + 1.0 / (k + 1)) / (fk * fk1);
        T.af[k] = (float)T.a[k];
        T.bf[k] = (float)T.b[k];
        T.cf_[k] = (float)T.c[k];
        T.df[k] = (float)T.d[k];
    }
    return T;
}

void upload_lag_rule_p2p() {
    upload_lag_rule_local();
    SeriesTab T = make_series_tab();
    CFMM_CUDA(cudaMemcpyToSymbol(c_ser, &T, sizeof(T)));
}

// number of series terms for |q|^2 = aq, FP64 (truncation below 1e-18)
__device__ __forceinline__ int series_terms64(double aq) {
    return aq <= 0.0625 ? 8 : aq <= 1.0 ? 11 : aq <= 5.0625 ? 14 : aq <= 16.0 ? 16 : 21;
}
// FP32 (truncation below 1e-9)
__device__ __forceinline__ int series_terms32(float aq) {
    return aq <= 0.0625f ? 5 : aq <= 1.0f ? 7 : aq <= 5.0625f ? 9 : aq <= 16.0f ? 10 : 14;
}

// FP64 2D Helmholtz pair: returns SLP factor H0 and DLP factor kappa H1 / r
__device__ __forceinline__ void helm2d_pair64(cd r2, double kappa, bool slp, bool dlp, cd& h0, cd& g1) {
    const double kPi = 3.14159265358979323846, kG = 0.57721566490153286061;
    double k2 = kappa * kappa;
    cd q = (0.25 * k2) * r2;
    double aq = cabs2(q);
    if (aq <= 81.0) {
        cd w = -q;
        int K = series_terms64(aq);
        cd A = {c_ser.a[K], 0}, Bs = {c_ser.b[K], 0}, Cs = {c_ser.c[K], 0}, Ds = {c_ser.d[K], 0};
        for (int k = K - 1; k >= 0; --k) {
            A = A * w + cd{c_ser.a[k], 0};
            Cs = Cs * w + cd{c_ser.c[k], 0};
            if (dlp) {
                Bs = Bs * w + cd{c_ser.b[k], 0};
                Ds = Ds * w + cd{c_ser.d[k], 0};
            }
        }
        cd L = {0.25 * log(aq), 0.5 * atan2(q.y, q.x)};    // log(z/2)
        h0 = A + mul_i((2.0 / kPi) * ((L + cd{kG, 0}) * A - Cs));
        if (dlp) {
            cd ir2 = cinv(r2);
            cd y = (-2.0 / kPi) * ir2 + (k2 / kPi) * (L * Bs) - (k2 / (2.0 * kPi)) * Ds;
            g1 = (0.5 * k2) * Bs + mul_i(y);
        }
        return;
    }
    cd r = csqrt_p(r2);
    cd h1;
    hankel01(kappa * r, &h0, &h1);
    g1 = (kappa * h1) * cinv(r);
}

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
        if (slp) acc += cd{0.25 * log(cabs2(r2)), 0.5 * atan2(r2.y, r2.x)} * sg;
        if (dlp) acc -= (nd * cinv(r2)) * ta;
    } else if (DIM == 2) {
        cd h0, g1;
        helm2d_pair64(r2, kappa, slp, dlp, h0, g1);
        if (slp) acc += h0 * sg;
        if (dlp) acc += (g1 * nd) * ta;
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

// grad_x of K(x, y) sg + (n . grad_y K)(x, y) ta for one pair (d = x - y != 0),
// added to g[0..DIM-1] (Sec. 2.1: S' and D' are its normal components). With
// K = K(r): grad_x K = (K'/r) d and grad_x (n . grad_y K) = -(K'/r) n -
// ((K'' - K'/r)/r^2) (n.d) d.
template <int DIM, int KER>
__device__ __forceinline__ void pair_grad(const double* dr, const double* di, const double* nr, const double* ni,
                                          cd sg, cd ta, bool slp, bool dlp, double kappa, cd* g) {
    cd d[DIM];
    cd r2 = {0.0, 0.0};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        d[a] = cd{dr[a], di[a]};
        r2 += d[a] * d[a];
    }
    cd a1, a2;   // K'/r and (K'' - K'/r)/r^2
    if (DIM == 2 && KER == CFMM_LAPLACE) {
        cd ir2 = cinv(r2);
        a1 = ir2;
        a2 = -2.0 * (ir2 * ir2);
    } else if (DIM == 2) {
        cd r = csqrt_p(r2);
        cd h0, h1;
        hankel01(kappa * r, &h0, &h1);
        cd ir = cinv(r), ir2 = cinv(r2);
        a1 = (-kappa) * (h1 * ir);
        a2 = (-kappa * kappa * h0 + (2.0 * kappa) * (h1 * ir)) * ir2;
    } else if (KER == CFMM_LAPLACE) {
        cd r = csqrt_p(r2);
        cd ir = cinv(r), ir2 = cinv(r2);
        cd ir3 = ir * ir2;
        a1 = -ir3;
        a2 = 3.0 * (ir3 * ir2);
    } else {
        cd r = csqrt_p(r2);
        cd ir = cinv(r), ir2 = cinv(r2);
        cd e = cexp_i(kappa * r);
        cd ikr = mul_i(kappa * r);
        cd ir3 = ir * ir2;
        a1 = (e * (ikr - cd{1.0, 0.0})) * ir3;
        a2 = (e * (cd{3.0, 0.0} - 3.0 * ikr - (kappa * kappa) * r2)) * (ir3 * ir2);
    }
    cd cs = slp ? a1 * sg : cd{0, 0};
    cd cn = {0, 0}, cdd = {0, 0};
    if (dlp) {
        cd nd = {0.0, 0.0};
#pragma unroll
        for (int a = 0; a < DIM; ++a) nd += cd{nr[a], ni[a]} * d[a];
        cn = -(a1 * ta);
        cdd = -(a2 * (nd * ta));
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        cd v = (cs + cdd) * d[a];
        if (dlp) v += cn * cd{nr[a], ni[a]};
        g[a] += v;
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

// near-field gradient over List 1 (FP64); g = sorted gradient [rhs][DIM][n]
// (overwritten). Same staging and fixed-order combination as k_p2p.
template <int DIM, int KER>
__global__ void __launch_bounds__(kP2PThreads) k_p2p_grad(KParams K, const int* __restrict__ leaf_boxes,
                                                          const int* __restrict__ bst, const int* __restrict__ ben,
                                                          const int* __restrict__ l1off, const int* __restrict__ l1,
                                                          cd* __restrict__ g) {
    __shared__ SrcTile S;
    __shared__ cd red[kP2PThreads];
    const int64_t n = K.n_src;
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
        cd acc[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) acc[a] = cd{0.0, 0.0};
        for (int q = l1off[b]; q < l1off[b + 1]; ++q) {
            int src = l1[q];
            int s0 = bst[src], s1 = ben[src];
            for (int c0 = s0; c0 < s1; c0 += kP2PChunk) {
                int cn = min(kP2PChunk, s1 - c0);
                __syncthreads();
                for (int j = threadIdx.x; j < cn; j += blockDim.x) {
                    int gi = c0 + j;
#pragma unroll
                    for (int a = 0; a < DIM; ++a) {
                        S.re[j][a] = K.src_re[a * n + gi];
                        S.im[j][a] = K.src_im[a * n + gi];
                        if (K.dlp) {
                            S.nr[j][a] = K.nrm_re[a * n + gi];
                            S.ni[j][a] = K.nrm_im[a * n + gi];
                        }
                    }
                    if (K.slp) S.sg[j] = K.sigma[(int64_t)rhs * K.dens_stride + gi];
                    if (K.dlp) S.ta[j] = K.tau[(int64_t)rhs * K.dens_stride + gi];
                }
                __syncthreads();
                if (!tvalid) continue;
                for (int j = split; j < cn; j += kP2PSplit) {
                    double dr[DIM], di[DIM];
                    bool zero = true;
#pragma unroll
                    for (int a = 0; a < DIM; ++a) {
                        dr[a] = xr[a] - S.re[j][a];
                        di[a] = xim[a] - S.im[j][a];
                        zero = zero && dr[a] == 0.0 && di[a] == 0.0;
                    }
                    if (zero) continue;
                    pair_grad<DIM, KER>(dr, di, S.nr[j], S.ni[j], K.slp ? S.sg[j] : cd{0, 0},
                                        K.dlp ? S.ta[j] : cd{0, 0}, K.slp, K.dlp, K.kappa, acc);
                }
            }
        }
        cd* gout = g + (int64_t)rhs * DIM * K.n_trg + ti;
#pragma unroll
        for (int a = 0; a < DIM; ++a)
            finish_target<DIM, KER>(acc[a], red, tl, split, tvalid, gout + (int64_t)a * K.n_trg, false);
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

// ---------------------------------------------------------------------------
// Mixed precision (complex64 kernel arithmetic, compensated FP32 sums).
// Coordinates enter as FP64 offsets from a reference point of the target
// block (the first target), split into FP32 hi + lo parts; the pair
// difference (x_h - y_h) + (x_l - y_l) keeps FP32 relative accuracy even for
// near-coincident pairs (Sterbenz: x_h - y_h is exact when x_h, y_h are
// close). Sums over sources use compensated (Kahan) FP32 accumulation; the
// few partial sums of a target are combined in FP64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void helm2d_pair32(cf r2, float kappa, bool dlp, cf& h0, cf& g1) {
    const float kPi = 3.14159265f, kG = 0.5772156649f;
    float k2 = kappa * kappa;
    cf q = (0.25f * k2) * r2;
    float aq = q.x * q.x + q.y * q.y;
    cf w = cf{-q.x, -q.y};
    int K = series_terms32(aq);
    cf A = {c_ser.af[K], 0.f}, Bs = {c_ser.bf[K], 0.f}, Cs = {c_ser.cf_[K], 0.f}, Ds = {c_ser.df[K], 0.f};
    for (int k = K - 1; k >= 0; --k) {
        A = A * w + cf{c_ser.af[k], 0.f};
        Cs = Cs * w + cf{c_ser.cf_[k], 0.f};
        if (dlp) {
            Bs = Bs * w + cf{c_ser.bf[k], 0.f};
            Ds = Ds * w + cf{c_ser.df[k], 0.f};
        }
    }
    cf L = {0.25f * logf(aq), 0.5f * atan2f(q.y, q.x)};
    cf lg = L + cf{kG, 0.f};
    h0 = A + mul_if((2.f / kPi) * (lg * A - Cs));
    if (dlp) {
        cf ir2 = cinvf(r2);
        cf y = (-2.f / kPi) * ir2 + (k2 / kPi) * (L * Bs) - (k2 / (2.f * kPi)) * Ds;
        g1 = (0.5f * k2) * Bs + mul_if(y);
    }
}

// Error-free transformations (Dekker, Knuth): the product and sum of two
// floats as an unevaluated hi + lo pair.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = a * b;
    e = fmaf(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// (h1 + l1) * (h2 + l2) added to the double-float accumulator (S, E)
__device__ __forceinline__ void df_fma(float h1, float l1, float h2, float l2, float sgn, float& S, float& E) {
    float p, e, t;
    two_prod(h1, h2, p, e);
    e = fmaf(h1, l2, fmaf(l1, h2, e));
    two_sum(S, sgn * p, S, t);
    E += t + sgn * e;
}

// n . d with the normal and the difference each as FP32 hi + lo: on a smooth
// curve or surface n is nearly orthogonal to d for close pairs, so n . d
// cancels; the double-float evaluation keeps its FP32 relative accuracy.
template <int DIM>
__device__ __forceinline__ cf dot_nd(const float* dh_r, const float* dl_r, const float* dh_i, const float* dl_i,
                                     const float* nh_r, const float* nl_r, const float* nh_i, const float* nl_i) {
    float Sr = 0.f, Er = 0.f, Si = 0.f, Ei = 0.f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        df_fma(nh_r[a], nl_r[a], dh_r[a], dl_r[a], 1.f, Sr, Er);
        df_fma(nh_i[a], nl_i[a], dh_i[a], dl_i[a], -1.f, Sr, Er);
        df_fma(nh_r[a], nl_r[a], dh_i[a], dl_i[a], 1.f, Si, Ei);
        df_fma(nh_i[a], nl_i[a], dh_r[a], dl_r[a], 1.f, Si, Ei);
    }
    return cf{Sr + Er, Si + Ei};
}

// The hi/lo parts of a target and a source (offsets from the block's
// reference point), for pairs that need the difference in FP64.
struct PairHL {
    const float *xhr, *xlr, *xhi, *xli;   // target
    const float *yhr, *ylr, *yhi, *yli;   // source
};

// r^2 in FP64 from the hi/lo parts (for |kappa r| beyond the complex64 range:
// the phase kappa*r needs more than FP32 relative accuracy there, and the
// FP32 difference of the hi parts is not exact for distant pairs)
template <int DIM>
__device__ __forceinline__ cd r2_from_hl(const PairHL& H) {
    cd r2 = {0.0, 0.0};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        cd d = {((double)H.xhr[a] - (double)H.yhr[a]) + ((double)H.xlr[a] - (double)H.ylr[a]),
                ((double)H.xhi[a] - (double)H.yhi[a]) + ((double)H.xli[a] - (double)H.yli[a])};
        r2 += d * d;
    }
    return r2;
}

// e^{i kappa r} and r for |kappa r| > 3 in double-float FP32 arithmetic (the
// FP32 phase would lose digits there): d = x - y as hi + lo per component
// (an exact two_sum of the hi parts plus the lo difference), r^2 in
// double-float, r = r0 + (r^2 - r0^2)/(2 r0) (one Newton step from the FP32
// root), kappa r in double-float, the phase reduced by 2 pi before sincosf.
template <int DIM>
__device__ __forceinline__ void far_phase_df(const PairHL& H, float kh, float kl, cf& e_ikr, cf& r) {
    float Sr = 0.f, Er = 0.f, Si = 0.f, Ei = 0.f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        float s, t, rh, rl, ih, il;
        two_sum(H.xhr[a], -H.yhr[a], s, t);
        two_sum(s, t + (H.xlr[a] - H.ylr[a]), rh, rl);
        two_sum(H.xhi[a], -H.yhi[a], s, t);
        two_sum(s, t + (H.xli[a] - H.yli[a]), ih, il);
        df_fma(rh, rl, rh, rl, 1.f, Sr, Er);
        df_fma(ih, il, ih, il, -1.f, Sr, Er);
        df_fma(rh, rl, ih, il, 2.f, Si, Ei);
    }
    cf r0 = csqrtf_p(cf{Sr + Er, Si + Ei});
    float Rr = Sr, ERr = Er, Ri = Si, ERi = Ei;
    df_fma(r0.x, 0.f, r0.x, 0.f, -1.f, Rr, ERr);
    df_fma(r0.y, 0.f, r0.y, 0.f, 1.f, Rr, ERr);
    df_fma(r0.x, 0.f, r0.y, 0.f, -2.f, Ri, ERi);
    cf corr = cf{Rr + ERr, Ri + ERi} * cinvf(2.f * r0);
    float th, te, dh, de;
    two_prod(kh, r0.x, th, te);
    te += fmaf(kh, corr.x, kl * r0.x);
    two_prod(kh, r0.y, dh, de);
    de += fmaf(kh, corr.y, kl * r0.y);
    const float kTwoPiH = 6.28318548202514648f;     // float(2 pi)
    const float kTwoPiL = -1.74845553e-07f;         // 2 pi - float(2 pi)
    float k = rintf(th * 0.159154943f);
    float q, qe;
    two_prod(k, kTwoPiH, q, qe);
    float red = (th - q) + ((te - qe) - k * kTwoPiL);
    float sn, cs;
    sincosf(red, &sn, &cs);
    float mag = expf(-dh) * (1.f - de);
    e_ikr = cf{mag * cs, mag * sn};
    r = r0 + corr;
}

template <int DIM, int KER>
__device__ __forceinline__ void pair_kernel32(const float* d_re, const float* d_im, const PairHL& H, cf nd, cf sg,
                                              cf ta, bool slp, bool dlp, float kappa, double kappa64, Kahan& acc) {
    cf d[DIM];
    cf r2 = {0.f, 0.f};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        d[a] = cf{d_re[a], d_im[a]};
        r2 = r2 + d[a] * d[a];
    }
    cf v = {0.f, 0.f};
    if (DIM == 2 && KER == CFMM_LAPLACE) {
        if (slp) v = cf{0.25f * logf(r2.x * r2.x + r2.y * r2.y), 0.5f * atan2f(r2.y, r2.x)} * sg;
        if (dlp) v = v - (nd * cinvf(r2)) * ta;
    } else if (DIM == 2) {
        float k2 = kappa * kappa;
        cf q = (0.25f * k2) * r2;
        // complex64 series only for |kappa r| <= 3 (|q| <= 2.25), where its
        // terms stay below ~1.3x the result; beyond, the FP64 evaluation
        if (q.x * q.x + q.y * q.y <= 5.0625f) {
            cf h0, g1;
            helm2d_pair32(r2, kappa, dlp, h0, g1);
            if (slp) v = h0 * sg;
            if (dlp) v = v + (g1 * nd) * ta;
        } else {
            // |kappa r| > 3: FP64 r^2 and the FP64 evaluation, result rounded to FP32
            cd h0, g1;
            helm2d_pair64(r2_from_hl<DIM>(H), kappa64, slp, dlp, h0, g1);
            if (slp) v = cf{(float)h0.x, (float)h0.y} * sg;
            if (dlp) v = v + (cf{(float)g1.x, (float)g1.y} * nd) * ta;
        }
    } else if (KER == CFMM_LAPLACE) {
        cf r = csqrtf_p(r2);
        cf ir = cinvf(r);
        if (slp) v = ir * sg;
        if (dlp) v = v + (nd * (ir * ir * ir)) * ta;
    } else {
        cf r = csqrtf_p(r2);
        cf g;
        float k4 = kappa * kappa * kappa * kappa;
        if (k4 * (r2.x * r2.x + r2.y * r2.y) <= 81.f) {    // |kappa r| <= 3
            float e = expf(-kappa * r.y), sn, cs;
            sincosf(kappa * r.x, &sn, &cs);
            g = cf{e * cs, e * sn} * cinvf(r);
        } else {
            // |kappa r| > 3: double-float phase
            cf e;
            far_phase_df<DIM>(H, kappa, (float)(kappa64 - (double)kappa), e, r);
            g = e * cinvf(r);
        }
        cf ir = cinvf(r);
        if (slp) v = g * sg;
        if (dlp) v = v + (nd * (cf{1.f, 0.f} - mul_if(kappa * r)) * g * (ir * ir)) * ta;
    }
    acc.add(v);
}

struct SrcTileF {
    float hr[kP2PChunk][3], lr[kP2PChunk][3], hi[kP2PChunk][3], li[kP2PChunk][3];
    float nhr[kP2PChunk][3], nlr[kP2PChunk][3], nhi[kP2PChunk][3], nli[kP2PChunk][3];
    cf sg[kP2PChunk], ta[kP2PChunk];
};

__device__ __forceinline__ void split_hl(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

template <int DIM, int KER>
__device__ void accumulate_sources32(SrcTileF& S, const KParams& K, int rhs, int s, int e, bool tvalid,
                                     const double* ref_re, const double* ref_im, const float* xh_r,
                                     const float* xl_r, const float* xh_i, const float* xl_i, Kahan& acc,
                                     int split) {
    const int64_t n = K.n_src;
    float kap = (float)K.kappa;
    for (int c0 = s; c0 < e; c0 += kP2PChunk) {
        int cn = min(kP2PChunk, e - c0);
        __syncthreads();
        for (int j = threadIdx.x; j < cn; j += blockDim.x) {
            int g = c0 + j;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                split_hl(K.src_re[a * n + g] - ref_re[a], S.hr[j][a], S.lr[j][a]);
                split_hl(K.src_im[a * n + g] - ref_im[a], S.hi[j][a], S.li[j][a]);
                if (K.dlp) {
                    split_hl(K.nrm_re[a * n + g], S.nhr[j][a], S.nlr[j][a]);
                    split_hl(K.nrm_im[a * n + g], S.nhi[j][a], S.nli[j][a]);
                }
            }
            if (K.slp) {
                cd v = K.sigma[(int64_t)rhs * K.dens_stride + g];
                S.sg[j] = cf{(float)v.x, (float)v.y};
            }
            if (K.dlp) {
                cd v = K.tau[(int64_t)rhs * K.dens_stride + g];
                S.ta[j] = cf{(float)v.x, (float)v.y};
            }
        }
        __syncthreads();
        if (tvalid) {
            for (int j = split; j < cn; j += kP2PSplit) {
                float dr[DIM], di[DIM], hr[DIM], lr[DIM], hi[DIM], li[DIM];
                bool zero = true;
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    hr[a] = xh_r[a] - S.hr[j][a];
                    lr[a] = xl_r[a] - S.lr[j][a];
                    hi[a] = xh_i[a] - S.hi[j][a];
                    li[a] = xl_i[a] - S.li[j][a];
                    zero = zero && hr[a] == 0.f && lr[a] == 0.f && hi[a] == 0.f && li[a] == 0.f;
                    dr[a] = hr[a] + lr[a];
                    di[a] = hi[a] + li[a];
                }
                if (zero) continue;
                cf nd = {0.f, 0.f};
                if (K.dlp) nd = dot_nd<DIM>(hr, lr, hi, li, S.nhr[j], S.nlr[j], S.nhi[j], S.nli[j]);
                PairHL H{xh_r, xl_r, xh_i, xl_i, S.hr[j], S.lr[j], S.hi[j], S.li[j]};
                pair_kernel32<DIM, KER>(dr, di, H, nd, K.slp ? S.sg[j] : cf{0, 0}, K.dlp ? S.ta[j] : cf{0, 0},
                                        K.slp, K.dlp, kap, K.kappa, acc);
            }
        }
    }
}

template <int DIM, int KER>
__device__ __forceinline__ void load_target32(const KParams& K, int ti, bool tvalid, const double* ref_re,
                                              const double* ref_im, float* xh_r, float* xl_r, float* xh_i,
                                              float* xl_i) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        double vr = tvalid ? K.trg_re[a * K.n_trg + ti] - ref_re[a] : 0.0;
        double vi = tvalid ? K.trg_im[a * K.n_trg + ti] - ref_im[a] : 0.0;
        split_hl(vr, xh_r[a], xl_r[a]);
        split_hl(vi, xh_i[a], xl_i[a]);
    }
}

template <int DIM, int KER>
__global__ void __launch_bounds__(kP2PThreads) k_p2p32(KParams K, const int* __restrict__ leaf_boxes,
                                                       const int* __restrict__ bst, const int* __restrict__ ben,
                                                       const int* __restrict__ l1off, const int* __restrict__ l1,
                                                       cd* __restrict__ out, int add) {
    __shared__ SrcTileF S;
    __shared__ cd red[kP2PThreads];
    int b = leaf_boxes[blockIdx.x];
    int rhs = blockIdx.y;
    int tl = threadIdx.x % kP2PTargets, split = threadIdx.x / kP2PTargets;
    int ts = bst[b], te = ben[b];
    double ref_re[DIM], ref_im[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        ref_re[a] = K.trg_re[a * K.n_trg + ts];
        ref_im[a] = K.trg_im[a * K.n_trg + ts];
    }
    for (int t0 = ts; t0 < te; t0 += kP2PTargets) {
        int ti = t0 + tl;
        bool tvalid = ti < te;
        float xh_r[DIM], xl_r[DIM], xh_i[DIM], xl_i[DIM];
        load_target32<DIM, KER>(K, ti, tvalid, ref_re, ref_im, xh_r, xl_r, xh_i, xl_i);
        Kahan acc;
        for (int q = l1off[b]; q < l1off[b + 1]; ++q) {
            int a = l1[q];
            accumulate_sources32<DIM, KER>(S, K, rhs, bst[a], ben[a], tvalid, ref_re, ref_im, xh_r, xl_r, xh_i,
                                           xl_i, acc, split);
        }
        finish_target<DIM, KER>(acc.value(), red, tl, split, tvalid, out + (int64_t)rhs * K.n_trg + ti, add != 0);
    }
}

template <int DIM, int KER>
__global__ void __launch_bounds__(kP2PThreads) k_direct32(KParams K, cd* __restrict__ out) {
    __shared__ SrcTileF S;
    __shared__ cd red[kP2PThreads];
    int rhs = blockIdx.y;
    int tl = threadIdx.x % kP2PTargets, split = threadIdx.x / kP2PTargets;
    int t0 = blockIdx.x * kP2PTargets;
    int ti = t0 + tl;
    bool tvalid = ti < K.n_trg;
    double ref_re[DIM], ref_im[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        ref_re[a] = K.trg_re[a * K.n_trg + t0];
        ref_im[a] = K.trg_im[a * K.n_trg + t0];
    }
    float xh_r[DIM], xl_r[DIM], xh_i[DIM], xl_i[DIM];
    load_target32<DIM, KER>(K, ti, tvalid, ref_re, ref_im, xh_r, xl_r, xh_i, xl_i);
    Kahan acc;
    accumulate_sources32<DIM, KER>(S, K, rhs, 0, (int)K.n_src, tvalid, ref_re, ref_im, xh_r, xl_r, xh_i, xl_i,
                                   acc, split);
    finish_target<DIM, KER>(acc.value(), red, tl, split, tvalid, out + (int64_t)rhs * K.n_trg + ti, false);
}

// ---------------------------------------------------------------------------
// Mixed-precision 3D Helmholtz near field on a power-of-two grid.
//
// Every coordinate v of a List-1 pair (real and imaginary parts, offsets from
// the target leaf's first point) is split as v = h + l with h = g rint(v/g)
// on a grid of step g = 2^e >= R/1024, R = 1.5 (k+1) w the per-axis reach of
// the near field of a leaf of width w at separation k (List-1 leaves differ
// by at most one level), and l = v - h, |l| <= g/2, rounded to FP32. Then the
// differences dh = x_h - y_h are multiples of g below 2048 g and are exact in
// FP32, as are their products and the sums of three of them (below 2^24 g^2):
//   r^2 = S_h + S_l,  S_h = sum dh_re^2 - dh_im^2 + 2 i dh_re dh_im  (exact),
//   S_l = sum (2 dh + dl) dl terms                           (FP32, small),
// so r^2 is known as an unevaluated FP32 pair to ~2^-24 g |r| absolute. The
// root r0 of the rounded sum is refined by one Newton step computed from
// that pair (r = r0 + (r^2 - r0^2)/(2 r0), with r0^2 formed by exact
// products), and kappa r is formed in double-float, so the phase and the
// decay exp(-kappa Im r) keep absolute errors near kappa g 2^-24 at any
// kappa r. The phase is reduced by 2 pi before sincosf. Sources are staged
// as float4 quadruples; the sum over sources is compensated (Kahan).
// ---------------------------------------------------------------------------
struct SrcTileG {
    float4 q0[kP2PChunk], q1[kP2PChunk], q2[kP2PChunk], dn[kP2PChunk];   // coordinates, densities
    float4 n0[kP2PChunk], n1[kP2PChunk], n2[kP2PChunk];                  // normals (double layer)
};

// v = h + l on the grid of step g (h exact in FP32 for |v| < 2^23 g)
__device__ __forceinline__ void split_grid(double v, double g, double ig, float& h, float& l) {
    double hv = g * rint(v * ig);
    h = (float)hv;
    l = (float)(v - hv);
}

// (re hi x3, im hi x3, re lo x3, im lo x3) <-> three float4
__device__ __forceinline__ void pack12(const float* a, float4& q0, float4& q1, float4& q2) {
    q0 = make_float4(a[0], a[1], a[2], a[3]);
    q1 = make_float4(a[4], a[5], a[6], a[7]);
    q2 = make_float4(a[8], a[9], a[10], a[11]);
}

// grid step for a target leaf of width w at separation k: 2^ceil(log2(R/1024))
__device__ __forceinline__ double near_grid_step(double w, int sep) {
    double R = 1.5 * (sep + 1) * w;
    int e;
    frexp(R / 1024.0, &e);     // R/1024 = f 2^e, f in [0.5, 1)
    return ldexp(1.0, e);
}

__global__ void __launch_bounds__(kP2PThreads) k_p2p32g_h3(KParams K, const int* __restrict__ leaf_boxes,
                                                           const int* __restrict__ bst, const int* __restrict__ ben,
                                                           const int* __restrict__ l1off,
                                                           const int* __restrict__ l1,
                                                           const int* __restrict__ blevel, double W, int sep,
                                                           cd* __restrict__ out, int add) {
    __shared__ SrcTileG S;
    __shared__ cd red[kP2PThreads];
    const int64_t n = K.n_src;
    int b = leaf_boxes[blockIdx.x];
    int rhs = blockIdx.y;
    int tl = threadIdx.x % kP2PTargets, split = threadIdx.x / kP2PTargets;
    int ts = bst[b], te = ben[b];
    double g = near_grid_step(ldexp(W, -blevel[b]), sep), ig = 1.0 / g;
    double ref_re[3], ref_im[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ref_re[a] = K.trg_re[a * K.n_trg + ts];
        ref_im[a] = K.trg_im[a * K.n_trg + ts];
    }
    const float kh = (float)K.kappa, kl = (float)(K.kappa - (double)kh);
    const float kTwoPiH = 6.28318548202514648f;     // float(2 pi)
    const float kTwoPiL = -1.74845553e-07f;         // 2 pi - float(2 pi)
    for (int t0 = ts; t0 < te; t0 += kP2PTargets) {
        int ti = t0 + tl;
        bool tvalid = ti < te;
        // target: x[0..2] re hi, x[3..5] im hi, x[6..8] re lo, x[9..11] im lo
        float x[12];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double vr = tvalid ? K.trg_re[a * K.n_trg + ti] - ref_re[a] : 0.0;
            double vi = tvalid ? K.trg_im[a * K.n_trg + ti] - ref_im[a] : 0.0;
            split_grid(vr, g, ig, x[a], x[6 + a]);
            split_grid(vi, g, ig, x[3 + a], x[9 + a]);
        }
        Kahan acc;
        for (int q = l1off[b]; q < l1off[b + 1]; ++q) {
            int src = l1[q];
            int s0 = bst[src], s1 = ben[src];
            for (int c0 = s0; c0 < s1; c0 += kP2PChunk) {
                int cn = min(kP2PChunk, s1 - c0);
                __syncthreads();
                for (int j = threadIdx.x; j < cn; j += blockDim.x) {
                    int gi = c0 + j;
                    float y[12];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        split_grid(K.src_re[a * n + gi] - ref_re[a], g, ig, y[a], y[6 + a]);
                        split_grid(K.src_im[a * n + gi] - ref_im[a], g, ig, y[3 + a], y[9 + a]);
                    }
                    pack12(y, S.q0[j], S.q1[j], S.q2[j]);
                    float4 dn = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (K.slp) {
                        cd v = K.sigma[(int64_t)rhs * K.dens_stride + gi];
                        dn.x = (float)v.x;
                        dn.y = (float)v.y;
                    }
                    if (K.dlp) {
                        cd v = K.tau[(int64_t)rhs * K.dens_stride + gi];
                        dn.z = (float)v.x;
                        dn.w = (float)v.y;
                        float nv[12];
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            split_hl(K.nrm_re[a * n + gi], nv[a], nv[6 + a]);
                            split_hl(K.nrm_im[a * n + gi], nv[3 + a], nv[9 + a]);
                        }
                        pack12(nv, S.n0[j], S.n1[j], S.n2[j]);
                    }
                    S.dn[j] = dn;
                }
                __syncthreads();
                if (!tvalid) continue;
                for (int j = split; j < cn; j += kP2PSplit) {
                    float4 a0 = S.q0[j], a1 = S.q1[j], a2 = S.q2[j];
                    // dh: re 0..2, im 0..2 (exact); dl likewise
                    float hr0 = x[0] - a0.x, hr1 = x[1] - a0.y, hr2 = x[2] - a0.z;
                    float hi0 = x[3] - a0.w, hi1 = x[4] - a1.x, hi2 = x[5] - a1.y;
                    float lr0 = x[6] - a1.z, lr1 = x[7] - a1.w, lr2 = x[8] - a2.x;
                    float li0 = x[9] - a2.y, li1 = x[10] - a2.z, li2 = x[11] - a2.w;
                    unsigned nz = (__float_as_uint(hr0) | __float_as_uint(hr1) | __float_as_uint(hr2) |
                                   __float_as_uint(hi0) | __float_as_uint(hi1) | __float_as_uint(hi2) |
                                   __float_as_uint(lr0) | __float_as_uint(lr1) | __float_as_uint(lr2) |
                                   __float_as_uint(li0) | __float_as_uint(li1) | __float_as_uint(li2)) &
                                  0x7fffffffu;
                    if (nz == 0u) continue;   // x == y: self pair / coincident point
                    // r^2 = (Srh + Srl) + i (Sih + Sil)
                    float Srh = hr0 * hr0;
                    Srh = fmaf(hr1, hr1, Srh);
                    Srh = fmaf(hr2, hr2, Srh);
                    Srh = fmaf(-hi0, hi0, Srh);
                    Srh = fmaf(-hi1, hi1, Srh);
                    Srh = fmaf(-hi2, hi2, Srh);
                    float Sih = hr0 * hi0;
                    Sih = fmaf(hr1, hi1, Sih);
                    Sih = fmaf(hr2, hi2, Sih);
                    Sih = 2.f * Sih;
                    float Srl = fmaf(2.f, hr0, lr0) * lr0;
                    Srl = fmaf(fmaf(2.f, hr1, lr1), lr1, Srl);
                    Srl = fmaf(fmaf(2.f, hr2, lr2), lr2, Srl);
                    Srl = fmaf(-fmaf(2.f, hi0, li0), li0, Srl);
                    Srl = fmaf(-fmaf(2.f, hi1, li1), li1, Srl);
                    Srl = fmaf(-fmaf(2.f, hi2, li2), li2, Srl);
                    float Sil = fmaf(hr0, li0, lr0 * (hi0 + li0));
                    Sil = fmaf(hr1, li1, fmaf(lr1, hi1 + li1, Sil));
                    Sil = fmaf(hr2, li2, fmaf(lr2, hi2 + li2, Sil));
                    Sil = 2.f * Sil;
                    float ra = Srh + Srl, rb = Sih + Sil;
                    // r0 = principal sqrt(ra + i rb) in FP32 (refined below)
                    float m = sqrtf(fmaf(ra, ra, rb * rb));
                    float t2 = 0.5f * (fabsf(ra) + m);
                    float rt = rsqrtf(t2);
                    float t = t2 * rt, u = 0.5f * rb * rt;
                    float a0r = ra >= 0.f ? t : fabsf(u);
                    float b0r = ra >= 0.f ? u : copysignf(t, rb);
                    // Newton step: delta = (r^2 - r0^2)/(2 r0), r0^2 from exact products
                    float p = a0r * a0r, e1 = fmaf(a0r, a0r, -p);
                    float qq = b0r * b0r, e2 = fmaf(b0r, b0r, -qq);
                    float hs, ls;
                    two_sum(p, -qq, hs, ls);
                    float dre = ((Srh - hs) - ls) + ((Srl - e1) + e2);
                    float pi_ = a0r * b0r, e3 = fmaf(a0r, b0r, -pi_);
                    float dim = ((Sih - 2.f * pi_) - 2.f * e3) + Sil;
                    float i2m = __fdividef(0.5f, m);
                    float der = fmaf(dre, a0r, dim * b0r) * i2m;
                    float dei = fmaf(dim, a0r, -dre * b0r) * i2m;
                    // kappa r in double-float: (th + te) + i (dh + de)
                    float th, tq, dh, dq;
                    two_prod(kh, a0r, th, tq);
                    tq = fmaf(kh, der, fmaf(kl, a0r, tq));
                    two_prod(kh, b0r, dh, dq);
                    dq = fmaf(kh, dei, fmaf(kl, b0r, dq));
                    float kk = rintf(th * 0.159154943f);
                    float q2, q2e;
                    two_prod(kk, kTwoPiH, q2, q2e);
                    float ph = (th - q2) + ((tq - q2e) - kk * kTwoPiL);
                    float sn, cs;
                    sincosf(ph, &sn, &cs);
                    float mag = expf(-dh) * (1.f - dq);
                    // 1/r with r = r0 + delta rounded to FP32
                    float rr = a0r + der, ri = b0r + dei;
                    float id = __frcp_rn(fmaf(rr, rr, ri * ri));
                    float irr = rr * id, iri = -ri * id;
                    cf gk = cf{mag * cs, mag * sn} * cf{irr, iri};   // e^{i kappa r}/r
                    float4 dn = S.dn[j];
                    cf v = {0.f, 0.f};
                    if (K.slp) v = gk * cf{dn.x, dn.y};
                    if (K.dlp) {
                        float4 b0 = S.n0[j], b1 = S.n1[j], b2 = S.n2[j];
                        const float dh_r[3] = {hr0, hr1, hr2}, dl_r[3] = {lr0, lr1, lr2};
                        const float dh_i[3] = {hi0, hi1, hi2}, dl_i[3] = {li0, li1, li2};
                        const float nh_r[3] = {b0.x, b0.y, b0.z}, nh_i[3] = {b0.w, b1.x, b1.y};
                        const float nl_r[3] = {b1.z, b1.w, b2.x}, nl_i[3] = {b2.y, b2.z, b2.w};
                        cf nd = dot_nd<3>(dh_r, dl_r, dh_i, dl_i, nh_r, nl_r, nh_i, nl_i);
                        cf ir = {irr, iri};
                        cf kr = {kh * rr, kh * ri};
                        v = v + (nd * (cf{1.f, 0.f} - mul_if(kr)) * gk * (ir * ir)) * cf{dn.z, dn.w};
                    }
                    acc.add(v);
                }
            }
        }
        finish_target<3, CFMM_HELMHOLTZ>(acc.value(), red, tl, split, tvalid, out + (int64_t)rhs * K.n_trg + ti,
                                        add != 0);
    }
}

template <int DIM, int KER>
static void launch_p2p_t(const KParams& K, const int* leaf_boxes, int nleaves, const int* bst, const int* ben,
                         const int* l1off, const int* l1, cd* out, int nrhs, bool add, bool mixed, cudaStream_t st) {
    if (nleaves == 0) return;
    dim3 grid(nleaves, nrhs);
    if (mixed) k_p2p32<DIM, KER><<<grid, kP2PThreads, 0, st>>>(K, leaf_boxes, bst, ben, l1off, l1, out, add ? 1 : 0);
    else k_p2p<DIM, KER><<<grid, kP2PThreads, 0, st>>>(K, leaf_boxes, bst, ben, l1off, l1, out, add ? 1 : 0);
    CFMM_LAUNCHED();
}

void launch_p2p(int dim, int ker, const KParams& K, const int* leaf_boxes, int nleaves, const int* bst,
                const int* ben, const int* l1off, const int* l1, cd* out, int nrhs, bool add, cudaStream_t st,
                bool mixed, const int* blevel, double W, int sep) {
    if (mixed && dim == 3 && ker == CFMM_HELMHOLTZ && blevel && nleaves > 0) {
        dim3 grid(nleaves, nrhs);
        k_p2p32g_h3<<<grid, kP2PThreads, 0, st>>>(K, leaf_boxes, bst, ben, l1off, l1, blevel, W, sep, out,
                                                  add ? 1 : 0);
        CFMM_LAUNCHED();
        return;
    }
    if (dim == 2 && ker == CFMM_LAPLACE) launch_p2p_t<2, CFMM_LAPLACE>(K, leaf_boxes, nleaves, bst, ben, l1off, l1, out, nrhs, add, mixed, st);
    else if (dim == 2) launch_p2p_t<2, CFMM_HELMHOLTZ>(K, leaf_boxes, nleaves, bst, ben, l1off, l1, out, nrhs, add, mixed, st);
    else if (ker == CFMM_LAPLACE) launch_p2p_t<3, CFMM_LAPLACE>(K, leaf_boxes, nleaves, bst, ben, l1off, l1, out, nrhs, add, mixed, st);
    else launch_p2p_t<3, CFMM_HELMHOLTZ>(K, leaf_boxes, nleaves, bst, ben, l1off, l1, out, nrhs, add, mixed, st);
}

template <int DIM, int KER>
static void launch_p2p_grad_t(const KParams& K, const int* leaf_boxes, int nleaves, const int* bst, const int* ben,
                              const int* l1off, const int* l1, cd* g, int nrhs, cudaStream_t st) {
    if (nleaves == 0) return;
    dim3 grid(nleaves, nrhs);
    k_p2p_grad<DIM, KER><<<grid, kP2PThreads, 0, st>>>(K, leaf_boxes, bst, ben, l1off, l1, g);
    CFMM_LAUNCHED();
}

void launch_p2p_grad(int dim, int ker, const KParams& K, const int* leaf_boxes, int nleaves, const int* bst,
                     const int* ben, const int* l1off, const int* l1, cd* g, int nrhs, cudaStream_t st) {
    if (dim == 2 && ker == CFMM_LAPLACE) launch_p2p_grad_t<2, CFMM_LAPLACE>(K, leaf_boxes, nleaves, bst, ben, l1off, l1, g, nrhs, st);
    else if (dim == 2) launch_p2p_grad_t<2, CFMM_HELMHOLTZ>(K, leaf_boxes, nleaves, bst, ben, l1off, l1, g, nrhs, st);
    else if (ker == CFMM_LAPLACE) launch_p2p_grad_t<3, CFMM_LAPLACE>(K, leaf_boxes, nleaves, bst, ben, l1off, l1, g, nrhs, st);
    else launch_p2p_grad_t<3, CFMM_HELMHOLTZ>(K, leaf_boxes, nleaves, bst, ben, l1off, l1, g, nrhs, st);
}

template <int DIM, int KER>
static void launch_direct_t(const KParams& K, cd* out, int nrhs, bool mixed, cudaStream_t st) {
    dim3 grid((unsigned)((K.n_trg + kP2PTargets - 1) / kP2PTargets), nrhs);
    if (mixed) k_direct32<DIM, KER><<<grid, kP2PThreads, 0, st>>>(K, out);
    else k_direct<DIM, KER><<<grid, kP2PThreads, 0, st>>>(K, out);
    CFMM_LAUNCHED();
}

void launch_direct(int dim, int ker, const KParams& K, cd* out, int nrhs, cudaStream_t st, bool mixed) {
    if (K.n_trg == 0) return;
    if (dim == 2 && ker == CFMM_LAPLACE) launch_direct_t<2, CFMM_LAPLACE>(K, out, nrhs, mixed, st);
    else if (dim == 2) launch_direct_t<2, CFMM_HELMHOLTZ>(K, out, nrhs, mixed, st);
    else if (ker == CFMM_LAPLACE) launch_direct_t<3, CFMM_LAPLACE>(K, out, nrhs, mixed, st);
    else launch_direct_t<3, CFMM_HELMHOLTZ>(K, out, nrhs, mixed, st);
}

}  // namespace cfmm
