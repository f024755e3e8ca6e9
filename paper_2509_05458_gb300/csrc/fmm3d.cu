// 3D complex-coordinate Laplace FMM: expansions and translations (Sec. 5.2,
// Sec. 6.4), FP64.
//
// Solid harmonics of a complex 3-vector x (x+ = x1 + i x2, x- = x1 - i x2,
// z = x3, rho^2 = x+ x- + z^2 = x.x):
//   regular   U_n^m = rho^n P_n^m(cos theta) e^{im phi}/(n+m)!
//   irregular T_n^m = (n-m)! P_n^m(cos theta) e^{im phi}/rho^{n+1}
// by their three-term recurrences (entire in x; no angle is formed);
// U_n^{-m} = (-1)^m U_n^m[x+ <-> x-], likewise T. With
//   1/|x - y| = sum (-1)^m U_n^{-m}(y) T_n^m(x)             (Lemma 5.2.1, Eq. sphaddition)
//   U_n^m(a + b) = sum U_k^l(a) U_{n-k}^{m-l}(b)
//   T_n^m(x - y) = sum (-1)^l U_k^{-l}(y) T_{n+k}^{m+l}(x)
// the operators are (coefficients at n*n + n + m):
//   P2M  M_n^m = sum s (-1)^m U_n^{-m}(y - c)          M2P  u = sum M_n^m T_n^m(x - c)
//   M2M  M_n^m(c) = sum (-1)^l U_k^l(c' - c) M_{n-k}^{m+l}(c')
//   M2L  L_k^l = (-1)^{k+l} sum M_n^m T_{n+k}^{m-l}(c_t - c_s)
//   L2L  L'_k^l = sum L_n^m U_{n-k}^{m-l}(c' - c)
//   P2L  L_k^l = sum s (-1)^l T_k^{-l}(y - c)          L2P  u = sum L_k^l U_k^l(x - c)
// The translations run as point-and-shoot (rotate the shift onto the z-axis,
// translate along it, rotate back; O(P^3)), in helm3d.cu's k_tr3l.
// Double layer: n.grad = nu+ d+ + nu- d- + n3 dz (nu+- = n1 +- i n2),
//   d+ U_n^m = -U_{n-1}^{m-1}/2, d- U_n^m = U_{n-1}^{m+1}/2, dz U_n^m = U_{n-1}^m,
//   d+ T_n^m = -T_{n+1}^{m-1}/2, d- T_n^m = T_{n+1}^{m+1}/2, dz T_n^m = -T_{n+1}^m.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "cfmm_special.cuh"
#include "kernels.cuh"

namespace cfmm {

__host__ __device__ __forceinline__ int nm_idx(int n, int m) { return n * n + n + m; }

// Table of U_n^m (reg = true) or T_n^m (reg = false), n <= P, of the complex
// 3-vector (a0, a1, a2), written to tab[nm_idx(n, m)]. Column m of each sign is
// computed by the threads t = lane0 .. in parallel (one column per thread).
__device__ void solid_table(bool reg, cd a0, cd a1, cd a2, int P, cd* tab, int t0, int nthreads) {
    cd xp = a0 + mul_i(a1), xm = a0 - mul_i(a1), z = a2;
    cd r2 = xp * xm + z * z;
    cd ir2 = {0, 0}, irho = {0, 0};
    if (!reg) {
        ir2 = cinv(r2);
        irho = cinv(csqrt_p(r2));
    }
    for (int col = t0; col < 2 * P + 1; col += nthreads) {
        int m = col <= P ? col : col - P;     // col 0..P: m >= 0 with x+; P+1..2P: m = 1..P with x-
        bool neg = col > P;
        cd xs = neg ? xm : xp;
        // diagonal value
        cd d;
        if (reg) {
            // U_m^m = (-x/2)^m / m!
            d = cd{1, 0};
            cd f = -0.5 * xs;
            for (int j = 1; j <= m; ++j) d = d * f * (1.0 / j);
        } else {
            // T_m^m = (-1)^m (2m-1)!! x^m / rho^{2m+1}
            d = irho;
            for (int j = 1; j <= m; ++j) d = d * (-(2.0 * j - 1.0)) * (xs * ir2);
        }
        double sg = (neg && (m & 1)) ? -1.0 : 1.0;
        tab[nm_idx(m, neg ? -m : m)] = sg * d;
        if (m + 1 > P) continue;
        cd p2 = d;
        cd p1 = reg ? z * d : (2.0 * m + 1.0) * (z * ir2) * d;
        tab[nm_idx(m + 1, neg ? -m : m)] = sg * p1;
        for (int n = m + 2; n <= P; ++n) {
            cd cur;
            if (reg) cur = ((2.0 * n - 1.0) * (z * p1) - r2 * p2) * (1.0 / ((n - m) * (double)(n + m)));
            else cur = ((2.0 * n - 1.0) * (z * p1) - ((double)(n - 1) * (n - 1) - (double)m * m) * p2) * ir2;
            tab[nm_idx(n, neg ? -m : m)] = sg * cur;
            p2 = p1;
            p1 = cur;
        }
    }
}

__device__ __forceinline__ cd tab_get(const cd* tab, int n, int m) {
    if (n < 0 || m > n || -m > n) return cd{0, 0};
    return tab[nm_idx(n, m)];
}

struct Exp3Args {
    const double* xr;
    const double* xi;
    const double* nr;
    const double* ni;
    int64_t n;
    const cd* sigma;
    const cd* tau;
    int64_t dstride;
    bool slp, dlp;
    const int* blevel;
    const int* bst;
    const int* ben;
    const double* cre;
    const double* cim;
    const int* Plev;
    const int64_t* eoff;
    int64_t ncoef;
};

__device__ __forceinline__ void load3(const double* re, const double* im, int64_t n, int64_t j, cd* x) {
    for (int a = 0; a < 3; ++a) x[a] = cd{re[a * n + j], im[a * n + j]};
}

// P2M (sing = 0) over a box's own points, or P2L (sing = 1) over its List-4 leaves.
// chunk sources at a time: their U (or T) tables in shared memory; each thread
// owns coefficients c and adds the sources' terms in source order.
__global__ void k_point_to_exp3(Exp3Args A, const int* __restrict__ boxes, const int* __restrict__ loff,
                                const int* __restrict__ lent, int sing, cd* __restrict__ out, int chunk) {
    extern __shared__ cd sm[];
    int b = boxes[blockIdx.x];
    int rhs = blockIdx.y;
    int P = A.Plev[A.blevel[b]];
    int nc = (P + 1) * (P + 1);
    int PT = sing ? P + 1 : P;                 // table order (P2L's dipole needs T_{k+1})
    int nt = (PT + 1) * (PT + 1);
    cd* acc = sm;
    cd* tabs = sm + nc;                        // [chunk][nt]
    cd* srcv = tabs + (size_t)chunk * nt;      // [chunk][6]: sigma, tau, nu+, nu-, n3
    for (int c = threadIdx.x; c < nc; c += blockDim.x) acc[c] = cd{0, 0};
    cd cen[3];
    for (int a = 0; a < 3; ++a) cen[a] = cd{A.cre[3 * b + a], A.cim[3 * b + a]};
    int qa = loff ? loff[b] : 0, qb = loff ? loff[b + 1] : 1;
    for (int q = qa; q < qb; ++q) {
        int src = loff ? lent[q] : b;
        int s0 = A.bst[src], s1 = A.ben[src];
        for (int c0 = s0; c0 < s1; c0 += chunk) {
            int cn = min(chunk, s1 - c0);
            __syncthreads();
            // tables: threads split (source, column)
            int cols = 2 * PT + 1;
            for (int w = threadIdx.x; w < cn * cols; w += blockDim.x) {
                int s = w / cols, col = w - s * cols;
                int64_t j = c0 + s;
                cd y[3];
                load3(A.xr, A.xi, A.n, j, y);
                solid_table(!sing, y[0] - cen[0], y[1] - cen[1], y[2] - cen[2], PT, tabs + (size_t)s * nt, col, cols);
                if (col == 0) {
                    cd* v = srcv + (size_t)s * 6;
                    v[0] = A.slp ? A.sigma[rhs * A.dstride + j] : cd{0, 0};
                    v[1] = A.dlp ? A.tau[rhs * A.dstride + j] : cd{0, 0};
                    if (A.dlp) {
                        cd nn[3];
                        load3(A.nr, A.ni, A.n, j, nn);
                        v[2] = nn[0] + mul_i(nn[1]);
                        v[3] = nn[0] - mul_i(nn[1]);
                        v[4] = nn[2];
                    }
                }
            }
            __syncthreads();
            for (int c = threadIdx.x; c < nc; c += blockDim.x) {
                int n = (int)sqrt((double)c);
                while (n * n > c) --n;
                while ((n + 1) * (n + 1) <= c) ++n;
                int m = c - n * n - n;
                double sg = (m & 1) ? -1.0 : 1.0;
                cd a = acc[c];
                for (int s = 0; s < cn; ++s) {
                    const cd* tb = tabs + (size_t)s * nt;
                    const cd* v = srcv + (size_t)s * 6;
                    cd term = {0, 0};
                    if (!sing) {
                        // (-1)^m [sigma U_n^{-m} + tau n.grad U_n^{-m}]
                        if (A.slp) term = v[0] * tb[nm_idx(n, -m)];
                        if (A.dlp) {
                            cd g = (-0.5 * v[2]) * tab_get(tb, n - 1, -m - 1) + (0.5 * v[3]) * tab_get(tb, n - 1, -m + 1) +
                                   v[4] * tab_get(tb, n - 1, -m);
                            term += v[1] * g;
                        }
                    } else {
                        // (-1)^l [sigma T_k^{-l} + tau n.grad T_k^{-l}]
                        if (A.slp) term = v[0] * tb[nm_idx(n, -m)];
                        if (A.dlp) {
                            cd g = (-0.5 * v[2]) * tab_get(tb, n + 1, -m - 1) + (0.5 * v[3]) * tab_get(tb, n + 1, -m + 1) -
                                   v[4] * tab_get(tb, n + 1, -m);
                            term += v[1] * g;
                        }
                    }
                    a += sg * term;
                }
                acc[c] = a;
            }
        }
    }
    __syncthreads();
    cd* o = out + (int64_t)rhs * A.ncoef + A.eoff[b];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        if (sing) o[c] += acc[c];
        else o[c] = acc[c];
    }
}

// M2P over List 3 and L2P: one thread per target; harmonics column by column
// in registers (no table)
__device__ cd eval_series(bool reg, cd a0, cd a1, cd a2, int P, const cd* coef) {
    cd xp = a0 + mul_i(a1), xm = a0 - mul_i(a1), z = a2;
    cd r2 = xp * xm + z * z;
    cd ir2 = {0, 0}, irho = {0, 0};
    if (!reg) {
        ir2 = cinv(r2);
        irho = cinv(csqrt_p(r2));
    }
    cd acc = {0, 0};
    for (int sgn = 0; sgn < 2; ++sgn) {
        cd xs = sgn ? xm : xp;
        cd d = reg ? cd{1, 0} : irho;
        for (int m = 0; m <= P; ++m) {
            if (m > 0) d = reg ? d * (-0.5 * xs) * (1.0 / m) : d * (-(2.0 * m - 1.0)) * (xs * ir2);
            if (sgn == 1 && m == 0) continue;
            double sg = (sgn && (m & 1)) ? -1.0 : 1.0;
            int mi = sgn ? -m : m;
            acc += sg * (d * coef[nm_idx(m, mi)]);
            if (m + 1 > P) continue;
            cd p2 = d;
            cd p1 = reg ? z * d : (2.0 * m + 1.0) * (z * ir2) * d;
            acc += sg * (p1 * coef[nm_idx(m + 1, mi)]);
            for (int n = m + 2; n <= P; ++n) {
                cd cur;
                if (reg) cur = ((2.0 * n - 1.0) * (z * p1) - r2 * p2) * (1.0 / ((n - m) * (double)(n + m)));
                else cur = ((2.0 * n - 1.0) * (z * p1) - ((double)(n - 1) * (n - 1) - (double)m * m) * p2) * ir2;
                acc += sg * (cur * coef[nm_idx(n, mi)]);
                p2 = p1;
                p1 = cur;
            }
        }
    }
    return acc;
}

// Target gradient of a solid-harmonic series: with d+ U_n^m = -U_{n-1}^{m-1}/2,
// d- U_n^m = U_{n-1}^{m+1}/2, dz U_n^m = U_{n-1}^m (L2P, reg) and d+ T_n^m =
// -T_{n+1}^{m-1}/2, d- T_n^m = T_{n+1}^{m+1}/2, dz T_n^m = -T_{n+1}^m (M2P),
// the derivatives of sum c_n^m H_n^m are series in H_{n'}^{m'} with shifted
// coefficients; one pass over H_{n'}^{m'}, n' <= Q (Q = P - 1 for L2P, P + 1
// for M2P), accumulates (dz, d+, d-). grad = (d+ + d-, i (d+ - d-), dz).
__device__ void eval_series_grad(bool reg, cd a0, cd a1, cd a2, int P, const cd* coef, cd& Dz, cd& Dp, cd& Dm) {
    cd xp = a0 + mul_i(a1), xm = a0 - mul_i(a1), z = a2;
    cd r2 = xp * xm + z * z;
    cd ir2 = {0, 0}, irho = {0, 0};
    if (!reg) {
        ir2 = cinv(r2);
        irho = cinv(csqrt_p(r2));
    }
    int Q = reg ? P - 1 : P + 1;
    int sh = reg ? 1 : -1;                       // coefficient order n' + sh
    auto c = [&](int n, int m) -> cd {
        if (n < 0 || n > P || m > n || -m > n) return cd{0, 0};
        return coef[nm_idx(n, m)];
    };
    Dz = Dp = Dm = cd{0, 0};
    auto add = [&](int n, int mi, cd h) {
        int k = n + sh;
        Dz += h * (reg ? c(k, mi) : -c(k, mi));
        Dp += h * (-0.5 * c(k, mi + 1));
        Dm += h * (0.5 * c(k, mi - 1));
    };
    if (Q < 0) return;
    for (int sgn = 0; sgn < 2; ++sgn) {
        cd xs = sgn ? xm : xp;
        cd d = reg ? cd{1, 0} : irho;
        for (int m = 0; m <= Q; ++m) {
            if (m > 0) d = reg ? d * (-0.5 * xs) * (1.0 / m) : d * (-(2.0 * m - 1.0)) * (xs * ir2);
            if (sgn == 1 && m == 0) continue;
            double sg = (sgn && (m & 1)) ? -1.0 : 1.0;
            int mi = sgn ? -m : m;
            add(m, mi, sg * d);
            if (m + 1 > Q) continue;
            cd p2 = d;
            cd p1 = reg ? z * d : (2.0 * m + 1.0) * (z * ir2) * d;
            add(m + 1, mi, sg * p1);
            for (int n = m + 2; n <= Q; ++n) {
                cd cur;
                if (reg) cur = ((2.0 * n - 1.0) * (z * p1) - r2 * p2) * (1.0 / ((n - m) * (double)(n + m)));
                else cur = ((2.0 * n - 1.0) * (z * p1) - ((double)(n - 1) * (n - 1) - (double)m * m) * p2) * ir2;
                add(n, mi, sg * cur);
                p2 = p1;
                p1 = cur;
            }
        }
    }
}

// target gradients of M2P (List 3) and L2P, FP64, added to g [rhs][3][n]
__global__ void k_eval3_grad(Exp3Args A, const int* __restrict__ leaves, const int* __restrict__ l3off,
                             const int* __restrict__ l3, const cd* __restrict__ mp, const cd* __restrict__ loc,
                             cd* __restrict__ g) {
    extern __shared__ cd sm[];
    int b = leaves[blockIdx.x];
    int rhs = blockIdx.y;
    int P = A.Plev[A.blevel[b]];
    cd* coef = sm;
    int s0 = A.bst[b], s1 = A.ben[b];
    for (int t0 = s0; t0 < s1; t0 += blockDim.x) {
        int i = t0 + threadIdx.x;
        bool valid = i < s1;
        cd x[3] = {{0, 0}, {0, 0}, {0, 0}};
        if (valid) load3(A.xr, A.xi, A.n, i, x);
        cd Dz = {0, 0}, Dp = {0, 0}, Dm = {0, 0};
        for (int q = l3off[b]; q < l3off[b + 1]; ++q) {
            int s = l3[q];
            int Ps = A.Plev[A.blevel[s]];
            __syncthreads();
            const cd* m = mp + (int64_t)rhs * A.ncoef + A.eoff[s];
            for (int c = threadIdx.x; c < (Ps + 1) * (Ps + 1); c += blockDim.x) coef[c] = m[c];
            __syncthreads();
            if (valid) {
                cd d[3];
                for (int a = 0; a < 3; ++a) d[a] = x[a] - cd{A.cre[3 * s + a], A.cim[3 * s + a]};
                cd z_, p_, m_;
                eval_series_grad(false, d[0], d[1], d[2], Ps, coef, z_, p_, m_);
                Dz += z_;
                Dp += p_;
                Dm += m_;
            }
        }
        __syncthreads();
        const cd* lc = loc + (int64_t)rhs * A.ncoef + A.eoff[b];
        for (int c = threadIdx.x; c < (P + 1) * (P + 1); c += blockDim.x) coef[c] = lc[c];
        __syncthreads();
        if (valid) {
            cd d[3];
            for (int a = 0; a < 3; ++a) d[a] = x[a] - cd{A.cre[3 * b + a], A.cim[3 * b + a]};
            cd z_, p_, m_;
            eval_series_grad(true, d[0], d[1], d[2], P, coef, z_, p_, m_);
            Dz += z_;
            Dp += p_;
            Dm += m_;
            cd* go = g + (int64_t)rhs * 3 * A.n + i;
            go[0] += Dp + Dm;
            go[A.n] += mul_i(Dp - Dm);
            go[2 * A.n] += Dz;
        }
    }
}

__global__ void k_eval3(Exp3Args A, const int* __restrict__ leaves, const int* __restrict__ l3off,
                        const int* __restrict__ l3, const cd* __restrict__ mp, const cd* __restrict__ loc,
                        cd* __restrict__ u, int maxP, int do_l2p) {
    extern __shared__ cd sm[];
    int b = leaves[blockIdx.x];
    int rhs = blockIdx.y;
    int P = A.Plev[A.blevel[b]];
    int nc = (P + 1) * (P + 1);
    cd* coef = sm;
    int s0 = A.bst[b], s1 = A.ben[b];
    for (int t0 = s0; t0 < s1; t0 += blockDim.x) {
        int i = t0 + threadIdx.x;
        bool valid = i < s1;
        cd x[3] = {{0, 0}, {0, 0}, {0, 0}};
        if (valid) load3(A.xr, A.xi, A.n, i, x);
        cd acc = {0, 0};
        for (int q = l3off[b]; q < l3off[b + 1]; ++q) {
            int s = l3[q];
            int Ps = A.Plev[A.blevel[s]];
            __syncthreads();
            const cd* m = mp + (int64_t)rhs * A.ncoef + A.eoff[s];
            for (int c = threadIdx.x; c < (Ps + 1) * (Ps + 1); c += blockDim.x) coef[c] = m[c];
            __syncthreads();
            if (valid) {
                cd d[3];
                for (int a = 0; a < 3; ++a) d[a] = x[a] - cd{A.cre[3 * s + a], A.cim[3 * s + a]};
                acc += eval_series(false, d[0], d[1], d[2], Ps, coef);
            }
        }
        if (!do_l2p) {
            // M2P only (the L2P runs in complex64): leaves without List 3 add nothing
            if (valid && l3off[b + 1] > l3off[b]) u[(int64_t)rhs * A.n + i] += acc;
            continue;
        }
        __syncthreads();
        const cd* lc = loc + (int64_t)rhs * A.ncoef + A.eoff[b];
        for (int c = threadIdx.x; c < nc; c += blockDim.x) coef[c] = lc[c];
        __syncthreads();
        if (valid) {
            cd d[3];
            for (int a = 0; a < 3; ++a) d[a] = x[a] - cd{A.cre[3 * b + a], A.cim[3 * b + a]};
            acc += eval_series(true, d[0], d[1], d[2], P, coef);
            u[(int64_t)rhs * A.n + i] += acc;
        }
    }
    (void)maxP;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Fmm3dState {
    int l0 = 1, nlev = 0, maxP = 0;
    std::vector<int> Plev;
    DevBuf<int> dPlev;
    DevBuf<int64_t> exp_off;
    int64_t ncoef = 0;
    std::vector<int> leaves_l0;
    DevBuf<int> d_leaves_l0;
    int n_p2l = 0;
    DevBuf<int> d_p2l_boxes;
    Lap3Tr* tr = nullptr;
    ~Fmm3dState() { lap3_tr_destroy(tr); }
};

static std::mutex g_mu3;
static std::vector<std::pair<cfmm_plan_s*, Fmm3dState*>>& exts3() {
    static std::vector<std::pair<cfmm_plan_s*, Fmm3dState*>> v;
    return v;
}
static Fmm3dState* state3(cfmm_plan_s* P) {
    std::lock_guard<std::mutex> lk(g_mu3);
    for (auto& e : exts3())
        if (e.first == P) return e.second;
    return nullptr;
}
void fmm3d_release(cfmm_plan_s* P) {
    std::lock_guard<std::mutex> lk(g_mu3);
    auto& v = exts3();
    for (size_t i = 0; i < v.size(); ++i)
        if (v[i].first == P) {
            delete v[i].second;
            v.erase(v.begin() + i);
            return;
        }
}

static int nterms_laplace3(int k, double eps) {
    double ratio = (std::sqrt(3.0) * 0.5) / (k + 0.5);
    double t = 1.0;
    int n = 0;
    for (;;) {
        ++n;
        t *= ratio;
        if (t <= eps) return n;
    }
}

constexpr int kExp3Threads = 128;
constexpr int kMax3Smem = 200 * 1024;

void fmm3d_setup(cfmm_plan_s* P) {
    TreeDev& T = P->tree;
    cudaStream_t st = P->stream;
    Fmm3dState* S = new Fmm3dState();
    {
        std::lock_guard<std::mutex> lk(g_mu3);
        exts3().push_back({P, S});
    }
    S->l0 = T.l0;
    S->nlev = T.nlevels;
    S->Plev.assign(T.nlevels, nterms_laplace3(P->sep, P->eps * 0.1));
    P->P = S->Plev;
    // 3D Helmholtz: the tree and lists are built; the apply reports that its
    // translations are not (unless the tree is a single leaf)
    if (T.nboxes <= 1 || P->kernel != CFMM_LAPLACE) return;
    int maxP = S->Plev[0];
    CFMM_REQUIRE(maxP <= 63, CFMM_EUNSUPPORTED, "3D Laplace: expansion order above 63 (eps too small)");
    S->maxP = maxP;
    S->dPlev.alloc(T.nlevels);
    CFMM_CUDA(cudaMemcpyAsync(S->dPlev.get(), S->Plev.data(), sizeof(int) * T.nlevels, cudaMemcpyHostToDevice, st));
    std::vector<int64_t> off(T.nboxes, -1);
    int64_t tot = 0;
    for (int l = S->l0; l < T.nlevels; ++l)
        for (int b = T.level_off[l]; b < T.level_off[l + 1]; ++b) {
            off[b] = tot;
            tot += (int64_t)(S->Plev[l] + 1) * (S->Plev[l] + 1);
        }
    S->ncoef = tot;
    P->ncoef = tot;
    S->exp_off.alloc(T.nboxes);
    CFMM_CUDA(cudaMemcpyAsync(S->exp_off.get(), off.data(), sizeof(int64_t) * T.nboxes, cudaMemcpyHostToDevice, st));
    std::vector<int> lvl(T.nboxes), l4(T.nboxes + 1), boxes;
    CFMM_CUDA(cudaMemcpyAsync(lvl.data(), T.level.get(), sizeof(int) * T.nboxes, cudaMemcpyDeviceToHost, st));
    CFMM_CUDA(cudaMemcpyAsync(l4.data(), T.loff[3].get(), sizeof(int) * (T.nboxes + 1), cudaMemcpyDeviceToHost, st));
    CFMM_CUDA(cudaStreamSynchronize(st));
    for (int b : T.leaf_boxes)
        if (lvl[b] >= S->l0) S->leaves_l0.push_back(b);
    S->d_leaves_l0.alloc(S->leaves_l0.size());
    CFMM_CUDA(cudaMemcpyAsync(S->d_leaves_l0.get(), S->leaves_l0.data(), sizeof(int) * S->leaves_l0.size(),
                              cudaMemcpyHostToDevice, st));
    for (int b = T.level_off[S->l0]; b < T.nboxes; ++b)
        if (l4[b + 1] > l4[b]) boxes.push_back(b);
    S->n_p2l = (int)boxes.size();
    S->d_p2l_boxes.alloc(boxes.size());
    if (!boxes.empty())
        CFMM_CUDA(cudaMemcpyAsync(S->d_p2l_boxes.get(), boxes.data(), sizeof(int) * boxes.size(),
                                  cudaMemcpyHostToDevice, st));
    CFMM_CUDA(cudaStreamSynchronize(st));
    for (auto f : {(const void*)k_point_to_exp3, (const void*)k_eval3, (const void*)k_eval3_grad})
        CFMM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax3Smem));
    S->tr = lap3_tr_create(P, maxP);
}

void fmm3d_apply(cfmm_plan_s* P, const cd* sigma, const cd* tau, int64_t dstride, cd* u, int nrhs, cd* g) {
    Fmm3dState* S = state3(P);
    CFMM_REQUIRE(S, CFMM_EINVAL, "plan has no 3D state");
    TreeDev& T = P->tree;
    cudaStream_t st = P->stream;
    auto rec = [&](int i) {
        if (P->timing) CFMM_CUDA(cudaEventRecord(P->ev[i], st));
    };
    KParams K{P->xr.get(), P->xi.get(), P->nr.get(), P->ni.get(), P->xr.get(), P->xi.get(), P->n, P->n,
              sigma, tau, dstride, P->slp, P->dlp, P->kappa};
    bool mixed = P->precision == CFMM_MIXED;
    CFMM_REQUIRE(T.nboxes <= 1 || P->kernel == CFMM_LAPLACE, CFMM_EUNSUPPORTED,
                 "3D Helmholtz translations are not built yet");
    if (T.nboxes <= 1) {
        for (int i = 2; i <= 6; ++i) rec(i);
        launch_p2p(3, P->kernel, K, T.d_leaf_boxes.get(), T.nleaves, T.start.get(), T.end.get(), T.loff[0].get(),
                   T.lent[0].get(), u, nrhs, false, st, mixed);
        if (g)
            launch_p2p_grad(3, P->kernel, K, T.d_leaf_boxes.get(), T.nleaves, T.start.get(), T.end.get(),
                            T.loff[0].get(), T.lent[0].get(), g, nrhs, st);
        rec(7);
        rec(8);
        return;
    }
    size_t need = (size_t)S->ncoef * nrhs;
    P->mpole.alloc(need);
    P->local.alloc(need);
    cd* mp = P->mpole.get();
    cd* lc = P->local.get();
    int maxP = S->maxP;
    Exp3Args A{P->xr.get(), P->xi.get(), P->nr.get(), P->ni.get(), P->n, sigma, tau, dstride, P->slp, P->dlp,
               T.level.get(), T.start.get(), T.end.get(), T.cen_re.get(), T.cen_im.get(), S->dPlev.get(),
               S->exp_off.get(), S->ncoef};
    auto p2x_smem = [&](int PT, int& chunk) {
        size_t nt = (size_t)(PT + 1) * (PT + 1);
        chunk = (int)std::max<size_t>(1, std::min<size_t>(16, (96 * 1024) / (nt * sizeof(cd))));
        return sizeof(cd) * ((size_t)(maxP + 1) * (maxP + 1) + (size_t)chunk * nt + (size_t)chunk * 6);
    };
    // (3) P2P (writes u) on the side stream, beside the far field
    {
        cudaStream_t ns = near_fork(P);
        launch_p2p(3, P->kernel, K, S->d_leaves_l0.get(), (int)S->leaves_l0.size(), T.start.get(), T.end.get(),
                   T.loff[0].get(), T.lent[0].get(), u, nrhs, false, ns, mixed);
        if (g)
            launch_p2p_grad(3, P->kernel, K, S->d_leaves_l0.get(), (int)S->leaves_l0.size(), T.start.get(),
                            T.end.get(), T.loff[0].get(), T.lent[0].get(), g, nrhs, ns);
    }
    near_launched(P);
    // (1) P2M (single layer: one lane per harmonic column; complex64 products
    // with FP64 sums in mixed precision)
    bool slp1 = P->slp && !P->dlp;
    bool p2m_done = slp1 && mixed &&
                    lap3_p2m32(S->tr, P, S->d_leaves_l0.get(), (int)S->leaves_l0.size(), maxP, S->dPlev.get(),
                               S->exp_off.get(), S->ncoef, sigma, dstride, mp, nrhs);
    if (!p2m_done && !(slp1 && lap3_p2m_slp(S->tr, P, S->d_leaves_l0.get(), (int)S->leaves_l0.size(), maxP,
                                            S->dPlev.get(), S->exp_off.get(), S->ncoef, sigma, dstride, mp, nrhs))) {
        int chunk;
        size_t smem = p2x_smem(maxP, chunk);
        dim3 g((unsigned)S->leaves_l0.size(), nrhs);
        if (g.x) {
            k_point_to_exp3<<<g, kExp3Threads, smem, st>>>(A, S->d_leaves_l0.get(), nullptr, nullptr, 0, mp, chunk);
            CFMM_LAUNCHED();
        }
    }
    rec(2);
    int Pu = S->Plev[0];
    // (2) M2M
    for (int l = T.nlevels - 2; l >= S->l0; --l)
        lap3_tr_launch(S->tr, P, 0, l, Pu, S->exp_off.get(), S->ncoef, mp, mp, nrhs);
    rec(3);
    // (4) M2L
    for (int l = S->l0; l < T.nlevels; ++l)
        lap3_tr_launch(S->tr, P, 1, l, Pu, S->exp_off.get(), S->ncoef, mp, lc, nrhs);
    rec(4);
    // (6) P2L
    if (S->n_p2l > 0) {
        int chunk;
        size_t smem = p2x_smem(maxP + 1, chunk);
        dim3 g(S->n_p2l, nrhs);
        k_point_to_exp3<<<g, kExp3Threads, smem, st>>>(A, S->d_p2l_boxes.get(), T.loff[3].get(), T.lent[3].get(), 1,
                                                       lc, chunk);
        CFMM_LAUNCHED();
    }
    rec(5);
    // (7) L2L
    for (int l = S->l0 + 1; l < T.nlevels; ++l)
        lap3_tr_launch(S->tr, P, 2, l, Pu, S->exp_off.get(), S->ncoef, lc, lc, nrhs);
    rec(6);
    rec(7);
    near_join(P);   // the near field has written u
    // (5) M2P, (8) L2P (complex64 in mixed precision)
    {
        dim3 gr((unsigned)S->leaves_l0.size(), nrhs);
        k_eval3<<<gr, kExp3Threads, sizeof(cd) * (size_t)(maxP + 1) * (maxP + 1), st>>>(A, S->d_leaves_l0.get(), T.loff[2].get(), T.lent[2].get(),
                                                          mp, lc, u, maxP, mixed ? 0 : 1);
        CFMM_LAUNCHED();
        if (mixed) lap3_l2p32(S->tr, P, S->d_leaves_l0.get(), (int)S->leaves_l0.size(), maxP, S->dPlev.get(),
                              S->exp_off.get(), S->ncoef, lc, u, nrhs);
        if (g && gr.x) {
            k_eval3_grad<<<gr, kExp3Threads, sizeof(cd) * (size_t)(maxP + 1) * (maxP + 1), st>>>(
                A, S->d_leaves_l0.get(), T.loff[2].get(), T.lent[2].get(), mp, lc, g);
            CFMM_LAUNCHED();
        }
    }
    rec(8);
}

}  // namespace cfmm
