// 2D complex-coordinate FMM: expansions and translations (Sec. 4, Sec. 6.4).
//
// Notation: for a complex displacement d = (d1, d2) put zeta = d1 + i d2,
// eta = d1 - i d2 (r^2 = zeta*eta, e^{+-i phi} = zeta/r, eta/r; Def. 3.1).
//
// 2D Laplace (Sec. 4.2) -- coefficient layout [c0, c_1..c_P, c_{P+1}..c_{2P}]:
//   multipole  u = M0 log r + sum Mp_n eta^-n + sum Mm_n zeta^-n
//              Mp_n = -(1/2n) sum eta_j^n s_j ;  Mm_n likewise in zeta
//   local      u = L0 + sum Lp_n zeta^n + sum Lm_n eta^n
//   M2M/M2L/L2L: the binomial re-expansions of Lemma 4.2.4 in zeta and eta
//   separately; the M0 term of M2L is -(1/2k) zeta0^-k M0 (derived from
//   log(1 - z) = -sum z^k/k).
// 2D Helmholtz (Sec. 4.3) -- layout [c_{-P} .. c_P]: with
//   G_n(d) = J_n(kappa r) e^{in phi}, S_n(d) = H_n^(1)(kappa r) e^{in phi}
//   and Graf's theorem (Thm 3.2.1): for expansions about c re-centred at c',
//   P2M  M_n = sum G_{-n}(c - y) s      M2P  u = sum M_n S_n(x - c)
//   M2M  M'_m = sum G_{n-m}(c' - c) M_n M2L  L_j = sum S_{n-j}(c' - c) M_n
//   L2L  L'_m = sum G_{n-m}(c' - c) L_n P2L  L_j = sum S_{-j}(c' - y) s
//   L2P  u = sum L_n G_n(x - c').
// Double layer: source-side terms differentiated along the caller's normal,
//   n.grad_y = nu d/dzeta + nut d/deta (nu = n1 + i n2, nut = n1 - i n2),
//   d/dzeta G_n = (kappa/2) G_{n-1}, d/deta G_n = -(kappa/2) G_{n+1}.
//
// Helmholtz translation tables depend only on the geometry and are built
// once per plan (one table per List-2 pair and per child box).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <mutex>

#include "cfmm_special.cuh"
#include "kernels.cuh"

namespace cfmm {

void upload_lag_rule_fmm2d() { upload_lag_rule_local(); }

constexpr int kExpThreads = 64;
constexpr int kMaxSmem = 200 * 1024;

// per-plan constants of the 2D expansions
struct Fmm2dState {
    int ker;
    int l0, nlev;
    std::vector<int> Plev;                 // host
    DevBuf<int> dPlev;
    DevBuf<int64_t> exp_off;               // per box (coefficient offset), -1 below l0
    int64_t ncoef = 0;
    int maxP = 0;
    // Laplace: binomial table C(n, k), n, k <= NB
    int NB = 0;
    DevBuf<double> binom;
    // Helmholtz translation tables
    DevBuf<cd> t_m2l;                      // per List-2 entry: S_j(c_t - c_s), j = -2P..2P
    std::vector<int64_t> m2l_base;         // per level: table base (complex units)
    std::vector<int> m2l_q0;               // per level: first List-2 entry index
    DevBuf<int64_t> d_m2l_base;
    DevBuf<int> d_m2l_q0;
    DevBuf<cd> t_shift;                    // per child box: G_j(c_parent - c_child), j = -(Pc+Pp)..(Pc+Pp)
    // Helmholtz: per point, the regular row T_m(c - y), m = -P-1..P+1 (P of
    // the point's leaf, index m + P + 1, stride RL), c its leaf's centre; P2M
    // of the leaf and L2P at the point both use it (geometry only)
    DevBuf<cd> lrow;
    int RL = 0;
    DevBuf<int64_t> shift_off;             // per box, -1 when none
    // work lists
    std::vector<int> leaves_l0;            // leaves at level >= l0
    DevBuf<int> d_leaves_l0;
    int maxP_leaf = 0;                     // largest order at a leaf level (P2M)
    int maxP_fine = 0;                     // largest order at or below the coarsest leaf level (M2P, L2P)
    bool rows_side = false;                // the row table is being built on the side stream
    int n_p2l = 0;                         // boxes with a non-empty List 4
    DevBuf<int> d_p2l_boxes;
    // Helmholtz M2L work split: chunks of at most kM2LChunk List-2 entries
    std::vector<int> lvl_chunk0;           // per level: first chunk (levels >= l0), size nlev+1
    std::vector<int64_t> lvl_part0;        // per level: first partial-sum slot (complex units)
    DevBuf<int> chunk_box, chunk_q0, chunk_q1, box_chunk0;   // box_chunk0: [nboxes+1]
    int64_t npart = 0;                     // partial-sum slots per rhs
    DevBuf<cd> part;
};


// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void zeta_eta(cd d0, cd d1, cd& z, cd& e) {
    z = d0 + mul_i(d1);
    e = d0 - mul_i(d1);
}

__device__ __forceinline__ cd load_pt(const double* a, int64_t n, int axis, int64_t i) { return cd{a[axis * n + i], 0}; }

// Fill row[0 .. 2P+2] with T_m(d), m = -P-1..P+1 (index m + P + 1), where
// T = G (kind 0, regular) or S (kind 1, singular) of the displacement d.
__device__ void cyl_row(int kind, cd zeta, cd eta, double kappa, int P, cd* row) {
    cd r2 = zeta * eta;
    cd r = csqrt_p(r2);
    int M = P + 1;
    cd* pos = row + M;   // pos[m] = T_m for m >= 0
    if (kind == 0) {
        if (r.x == 0.0 && r.y == 0.0) {
            for (int m = -M; m <= M; ++m) row[m + M] = cd{m == 0 ? 1.0 : 0.0, 0.0};
            return;
        }
        bessel_j_seq(kappa * r, M, pos);
    } else {
        cd h0, h1;
        cd z = kappa * r;
        hankel01(z, &h0, &h1);
        pos[0] = h0;
        if (M >= 1) pos[1] = h1;
        cd zi = cinv(z);
        for (int m = 1; m < M; ++m) pos[m + 1] = rmac(-pos[m - 1], 2.0 * m, zi * pos[m]);
    }
    cd ir = cinv(r);
    cd u = zeta * ir, v = eta * ir;
    cd up = u, vp = v;
    for (int m = 1; m <= M; ++m) {
        cd f = pos[m];
        cd neg = (m & 1) ? -f : f;
        row[M - m] = neg * vp;
        pos[m] = f * up;
        up = up * u;
        vp = vp * v;
    }
}

// Regular rows of every point about its leaf's centre (plan time): block per
// leaf, thread per point.
__global__ void k_leaf_rows(const int* __restrict__ leaves, const int* __restrict__ blevel,
                            const int* __restrict__ bst, const int* __restrict__ ben, const int* __restrict__ Plev,
                            const double* __restrict__ xr, const double* __restrict__ xi, int64_t n,
                            const double* __restrict__ cre, const double* __restrict__ cim, double kappa, int RL,
                            cd* __restrict__ lrow) {
    int b = leaves[blockIdx.x];
    int P = Plev[blevel[b]];
    cd cen0 = {cre[2 * b], cim[2 * b]}, cen1 = {cre[2 * b + 1], cim[2 * b + 1]};
    for (int j = bst[b] + threadIdx.x; j < ben[b]; j += blockDim.x) {
        cd y0 = {xr[j], xi[j]}, y1 = {xr[n + j], xi[n + j]};
        cd z, e;
        zeta_eta(cen0 - y0, cen1 - y1, z, e);   // D = c - y
        cyl_row(0, z, e, kappa, P, lrow + (int64_t)j * RL);
    }
}

// ---------------------------------------------------------------------------
// P2M (step 1) and P2L (step 6): point terms reduced per coefficient
// ---------------------------------------------------------------------------
struct ExpArgs {
    const double* xr;
    const double* xi;
    const double* nr;
    const double* ni;
    int64_t n;
    const cd* sigma;
    const cd* tau;
    int64_t dstride;
    bool slp, dlp;
    double kappa;
    const int* blevel;
    const int* bst;
    const int* ben;
    const double* cre;
    const double* cim;
    const int* Plev;
    const int64_t* eoff;
    int64_t ncoef;
};

// term row (Laplace) for a source at d = y - c, regular (P2M) or singular (P2L)
__device__ void lap_terms(bool sing, cd zeta, cd eta, cd s, cd t, cd nu, cd nut, int P, bool slp, bool dlp,
                          cd* row) {
    if (!sing) {
        row[0] = slp ? s : cd{0, 0};
        cd ep = {1, 0}, zp = {1, 0};
        for (int k = 1; k <= P; ++k) {
            cd a = {0, 0}, b = {0, 0};
            if (slp) {
                a = (-0.5 / k) * (ep * eta) * s;
                b = (-0.5 / k) * (zp * zeta) * s;
            }
            if (dlp) {
                a -= 0.5 * (nut * ep) * t;
                b -= 0.5 * (nu * zp) * t;
            }
            row[k] = a;
            row[P + k] = b;
            ep = ep * eta;
            zp = zp * zeta;
        }
    } else {
        cd iz = cinv(zeta), ie = cinv(eta);
        cd v0 = {0, 0};
        if (slp) v0 = (0.5 * clog_p(zeta * eta)) * s;
        if (dlp) v0 += (0.5 * (nu * iz + nut * ie)) * t;
        row[0] = v0;
        cd zp = iz, ep = ie;   // zeta^-k, eta^-k
        for (int k = 1; k <= P; ++k) {
            cd a = {0, 0}, b = {0, 0};
            if (slp) {
                a = (-0.5 / k) * zp * s;
                b = (-0.5 / k) * ep * s;
            }
            if (dlp) {
                a += 0.5 * (nu * (zp * iz)) * t;
                b += 0.5 * (nut * (ep * ie)) * t;
            }
            row[k] = a;
            row[P + k] = b;
            zp = zp * iz;
            ep = ep * ie;
        }
    }
}

// One CTA per target box; sources = the box's own points (P2M, list == null)
// or the points of the List-4 leaves (P2L). Result added to (P2L) or stored
// in (P2M) out[rhs][eoff[b] + c].
template <int KER>
__global__ void k_point_to_exp(ExpArgs A, const int* __restrict__ boxes, const int* __restrict__ loff,
                               const int* __restrict__ lent, int sing, cd* __restrict__ out, int chunk,
                               const cd* __restrict__ lrow, int RL) {
    extern __shared__ cd sm[];
    int b = boxes[blockIdx.x];
    int rhs = blockIdx.y;
    int P = A.Plev[A.blevel[b]];
    int nc = 2 * P + 1;
    int R = KER == CFMM_LAPLACE ? nc : nc + 2;
    cd* acc = sm;
    cd* rows = sm + nc;
    cd* wts = rows + (size_t)chunk * R;        // Helmholtz: per source (s, -k/2 nu t, k/2 nu~ t)
    for (int c = threadIdx.x; c < nc; c += blockDim.x) acc[c] = cd{0, 0};
    cd cen0 = {A.cre[2 * b], A.cim[2 * b]}, cen1 = {A.cre[2 * b + 1], A.cim[2 * b + 1]};
    int qa = loff ? loff[b] : 0, qb = loff ? loff[b + 1] : 1;
    for (int q = qa; q < qb; ++q) {
        int src = loff ? lent[q] : b;
        int s0 = A.bst[src], s1 = A.ben[src];
        for (int c0 = s0; c0 < s1; c0 += chunk) {
            int cn = min(chunk, s1 - c0);
            __syncthreads();
            if (threadIdx.x < cn) {
                int64_t j = c0 + threadIdx.x;
                cd y0 = {A.xr[j], A.xi[j]}, y1 = {A.xr[A.n + j], A.xi[A.n + j]};
                cd s = A.slp ? A.sigma[rhs * A.dstride + j] : cd{0, 0};
                cd t = A.dlp ? A.tau[rhs * A.dstride + j] : cd{0, 0};
                cd nu = {0, 0}, nut = {0, 0};
                if (A.dlp) {
                    cd n0 = {A.nr[j], A.ni[j]}, n1 = {A.nr[A.n + j], A.ni[A.n + j]};
                    nu = n0 + mul_i(n1);
                    nut = n0 - mul_i(n1);
                }
                cd* row = rows + (size_t)threadIdx.x * R;
                cd z, e;
                if (KER == CFMM_LAPLACE) {
                    zeta_eta(y0 - cen0, y1 - cen1, z, e);   // d = y - c
                    lap_terms(sing != 0, z, e, s, t, nu, nut, P, A.slp, A.dlp, row);
                } else {
                    if (lrow && !sing) {
                        // the plan's row of this point about its own leaf (this box)
                        const cd* src = lrow + j * RL;
                        for (int q = 0; q < R; ++q) row[q] = src[q];
                    } else {
                        zeta_eta(cen0 - y0, cen1 - y1, z, e);   // D = c - y
                        cyl_row(sing ? 1 : 0, z, e, A.kappa, P, row);
                    }
                    double hk = 0.5 * A.kappa;
                    cd* w = wts + 3 * threadIdx.x;
                    w[0] = s;
                    w[1] = (-hk) * (nu * t);
                    w[2] = hk * (nut * t);
                }
            }
            __syncthreads();
            for (int c = threadIdx.x; c < nc; c += blockDim.x) {
                cd a = acc[c];
                if (KER == CFMM_LAPLACE) {
                    for (int tt = 0; tt < cn; ++tt) a += rows[(size_t)tt * R + c];
                } else {
                    // coefficient n = c - P: s T_{-n} - (k/2)(nu T_{-n-1} - nu~ T_{-n+1}) t,
                    // T_k at row index k + P + 1
                    int i0 = 2 * P + 1 - c;
                    if (A.dlp) {
                        for (int tt = 0; tt < cn; ++tt) {
                            const cd* r = rows + (size_t)tt * R + i0;
                            const cd* w = wts + 3 * tt;
                            a = cmac(cmac(cmac(a, w[0], r[0]), w[1], r[-1]), w[2], r[1]);
                        }
                    } else {
                        for (int tt = 0; tt < cn; ++tt) a = cmac(a, wts[3 * tt], rows[(size_t)tt * R + i0]);
                    }
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

// ---------------------------------------------------------------------------
// M2M (step 2) and L2L (step 7): one CTA per target box at one level
// ---------------------------------------------------------------------------
struct TransArgs {
    const int* blevel;
    const int* parent;
    const int* cbeg;
    const int* cend;
    const double* cre;
    const double* cim;
    const int* Plev;
    const int64_t* eoff;
    int64_t ncoef;
    const double* binom;
    int NB;
    const cd* tshift;
    const int64_t* shoff;
};

__device__ __forceinline__ double binom_at(const TransArgs& T, int n, int k) { return T.binom[n * (T.NB + 1) + k]; }

// M2M: parent b gathers its children
template <int KER>
__global__ void k_m2m(TransArgs T, int lo, const cd* __restrict__ mp_in, cd* __restrict__ mp_out, const int* __restrict__ leaf) {
    extern __shared__ cd sm[];
    int b = lo + blockIdx.x;
    if (leaf[b]) return;
    int rhs = blockIdx.y;
    int Pp = T.Plev[T.blevel[b]];
    int ncp = 2 * Pp + 1;
    int Pc = T.Plev[T.blevel[b] + 1];      // every child sits one level finer
    int ncc = 2 * Pc + 1;
    cd* acc = sm;
    cd* src = sm + ncp;
    cd* pw = src + ncc;                    // Laplace: 2(Pp+1) powers; Helmholtz: 2(Pc+Pp)+1 table
    for (int c = threadIdx.x; c < ncp; c += blockDim.x) acc[c] = cd{0, 0};
    for (int ch = T.cbeg[b]; ch < T.cend[b]; ++ch) {
        __syncthreads();
        const cd* m = mp_in + (int64_t)rhs * T.ncoef + T.eoff[ch];
        for (int c = threadIdx.x; c < ncc; c += blockDim.x) src[c] = m[c];
        if (KER == CFMM_LAPLACE) {
            // powers of zeta0, eta0 of a = c_child - c_parent, up to Pp
            if (threadIdx.x == 0) {
                cd a0 = {T.cre[2 * ch] - T.cre[2 * b], T.cim[2 * ch] - T.cim[2 * b]};
                cd a1 = {T.cre[2 * ch + 1] - T.cre[2 * b + 1], T.cim[2 * ch + 1] - T.cim[2 * b + 1]};
                cd z, e;
                zeta_eta(a0, a1, z, e);
                cd zp = {1, 0}, ep = {1, 0};
                for (int k = 0; k <= Pp; ++k) {
                    pw[k] = zp;
                    pw[Pp + 1 + k] = ep;
                    zp = zp * z;
                    ep = ep * e;
                }
            }
        } else {
            const cd* tb = T.tshift + T.shoff[ch];
            int nt = 2 * (Pc + Pp) + 1;
            for (int c = threadIdx.x; c < nt; c += blockDim.x) pw[c] = tb[c];
        }
        __syncthreads();
        for (int c = threadIdx.x; c < ncp; c += blockDim.x) {
            cd a = acc[c];
            if (KER == CFMM_LAPLACE) {
                if (c == 0) {
                    a += src[0];
                } else {
                    bool isz = c > Pp;
                    int k = isz ? c - Pp : c;
                    const cd* pk = isz ? pw : pw + Pp + 1;      // zeta or eta powers
                    a += (-0.5 / k) * pk[k] * src[0];
                    int top = k < Pc ? k : Pc;
                    for (int nn = 1; nn <= top; ++nn) {
                        cd mn = isz ? src[Pc + nn] : src[nn];
                        a += binom_at(T, k - 1, k - nn) * (pk[k - nn] * mn);
                    }
                }
            } else {
                int m = c - Pp;
                int off = Pc + Pp;
                for (int nn = -Pc; nn <= Pc; ++nn) a = cmac(a, pw[nn - m + off], src[nn + Pc]);
            }
            acc[c] = a;
        }
    }
    __syncthreads();
    cd* o = mp_out + (int64_t)rhs * T.ncoef + T.eoff[b];
    for (int c = threadIdx.x; c < ncp; c += blockDim.x) o[c] = acc[c];
}

// L2L: child b (at level lo..) receives its parent's local expansion
template <int KER>
__global__ void k_l2l(TransArgs T, int lo, cd* __restrict__ loc) {
    extern __shared__ cd sm[];
    int b = lo + blockIdx.x;
    int rhs = blockIdx.y;
    int p = T.parent[b];
    int Pc = T.Plev[T.blevel[b]], Pp = T.Plev[T.blevel[p]];
    int ncc = 2 * Pc + 1, ncp = 2 * Pp + 1;
    cd* src = sm;
    cd* pw = sm + ncp;
    const cd* lp = loc + (int64_t)rhs * T.ncoef + T.eoff[p];
    for (int c = threadIdx.x; c < ncp; c += blockDim.x) src[c] = lp[c];
    if (KER == CFMM_LAPLACE) {
        if (threadIdx.x == 0) {
            // powers of -zeta0, -eta0 with a = c_parent - c_child
            cd a0 = {T.cre[2 * p] - T.cre[2 * b], T.cim[2 * p] - T.cim[2 * b]};
            cd a1 = {T.cre[2 * p + 1] - T.cre[2 * b + 1], T.cim[2 * p + 1] - T.cim[2 * b + 1]};
            cd z, e;
            zeta_eta(a0, a1, z, e);
            z = -z;
            e = -e;
            cd zp = {1, 0}, ep = {1, 0};
            for (int k = 0; k <= Pp; ++k) {
                pw[k] = zp;
                pw[Pp + 1 + k] = ep;
                zp = zp * z;
                ep = ep * e;
            }
        }
    } else {
        // table holds G_j(c_parent - c_child); L2L needs G_j(c_child - c_parent) = (-1)^j G_j(...)
        const cd* tb = T.tshift + T.shoff[b];
        int off = Pc + Pp;
        for (int c = threadIdx.x; c < 2 * off + 1; c += blockDim.x) {
            int j = c - off;
            pw[c] = (j & 1) ? -tb[c] : tb[c];
        }
    }
    __syncthreads();
    cd* o = loc + (int64_t)rhs * T.ncoef + T.eoff[b];
    for (int c = threadIdx.x; c < ncc; c += blockDim.x) {
        cd a = {0, 0};
        if (KER == CFMM_LAPLACE) {
            if (c == 0) {
                a = src[0];
                for (int nn = 1; nn <= Pp; ++nn) a += pw[nn] * src[nn] + pw[Pp + 1 + nn] * src[Pp + nn];
            } else {
                bool isz = c > Pc;
                int k = isz ? c - Pc : c;
                const cd* pk = isz ? pw + Pp + 1 : pw;          // Lm (eta) uses eta powers
                for (int nn = k; nn <= Pp; ++nn) {
                    cd ln = isz ? src[Pp + nn] : src[nn];
                    a += binom_at(T, nn, k) * (pk[nn - k] * ln);
                }
            }
        } else {
            int m = c - Pc;
            int off = Pc + Pp;
            for (int nn = -Pp; nn <= Pp; ++nn) a = cmac(a, pw[nn - m + off], src[nn + Pp]);
        }
        o[c] += a;
    }
}

// ---------------------------------------------------------------------------
// M2L (step 4) over List 2, all levels >= l0 in one launch
// ---------------------------------------------------------------------------
struct M2LArgs {
    const int* blevel;
    const double* cre;
    const double* cim;
    const int* Plev;
    const int64_t* eoff;
    int64_t ncoef;
    const int* loff;
    const int* lent;
    const double* binom;
    int NB;
    const cd* tab;
    const int64_t* tbase;
    const int* tq0;
};

__device__ __forceinline__ double binom_at_m2l(const M2LArgs& A, int n, int k) { return A.binom[n * (A.NB + 1) + k]; }

template <int KER>
__global__ void k_m2l(M2LArgs A, int first_box, const cd* __restrict__ mp, cd* __restrict__ loc) {
    extern __shared__ cd sm[];
    int b = first_box + blockIdx.x;
    int rhs = blockIdx.y;
    int l = A.blevel[b];
    int P = A.Plev[l];
    int nc = 2 * P + 1;
    cd* acc = sm;
    cd* src = sm + nc;
    cd* tb = src + nc;     // 4P+1 (Helmholtz) or 2*(2P+1) powers + log (Laplace)
    for (int c = threadIdx.x; c < nc; c += blockDim.x) acc[c] = cd{0, 0};
    for (int q = A.loff[b]; q < A.loff[b + 1]; ++q) {
        int s = A.lent[q];
        __syncthreads();
        const cd* m = mp + (int64_t)rhs * A.ncoef + A.eoff[s];
        for (int c = threadIdx.x; c < nc; c += blockDim.x) src[c] = m[c];
        if (KER == CFMM_LAPLACE) {
            // inverse powers of zeta0, eta0 (a = c_s - c_t), j = 0..2P, and log r0
            cd a0 = {A.cre[2 * s] - A.cre[2 * b], A.cim[2 * s] - A.cim[2 * b]};
            cd a1 = {A.cre[2 * s + 1] - A.cre[2 * b + 1], A.cim[2 * s + 1] - A.cim[2 * b + 1]};
            cd z, e;
            zeta_eta(a0, a1, z, e);
            cd iz = cinv(z), ie = cinv(e);
            for (int j = threadIdx.x; j <= 2 * P; j += blockDim.x) {
                // binary powering
                cd pz = {1, 0}, pe = {1, 0}, bz = iz, be = ie;
                int ee = j;
                while (ee) {
                    if (ee & 1) {
                        pz = pz * bz;
                        pe = pe * be;
                    }
                    bz = bz * bz;
                    be = be * be;
                    ee >>= 1;
                }
                tb[j] = pz;
                tb[2 * P + 1 + j] = pe;
            }
            if (threadIdx.x == 0) tb[4 * P + 2] = 0.5 * clog_p(z * e);
        } else {
            const cd* t = A.tab + A.tbase[l] + (int64_t)(q - A.tq0[l]) * (4 * P + 1);
            for (int c = threadIdx.x; c < 4 * P + 1; c += blockDim.x) tb[c] = t[c];
        }
        __syncthreads();
        for (int c = threadIdx.x; c < nc; c += blockDim.x) {
            cd a = acc[c];
            if (KER == CFMM_LAPLACE) {
                const cd* zi = tb;             // zeta0^-j
                const cd* ei = tb + 2 * P + 1; // eta0^-j
                if (c == 0) {
                    a += tb[4 * P + 2] * src[0];
                    for (int nn = 1; nn <= P; ++nn) {
                        cd t = ei[nn] * src[nn] + zi[nn] * src[P + nn];
                        a += (nn & 1) ? -t : t;
                    }
                } else {
                    bool ise = c > P;                 // Lm (eta) from Mp; Lp (zeta) from Mm
                    int k = ise ? c - P : c;
                    const cd* pk = ise ? ei : zi;
                    a += (-0.5 / k) * pk[k] * src[0];
                    for (int nn = 1; nn <= P; ++nn) {
                        cd mn = ise ? src[nn] : src[P + nn];
                        cd t = binom_at_m2l(A, nn + k - 1, k) * (pk[nn + k] * mn);
                        a += (nn & 1) ? -t : t;
                    }
                }
            } else {
                int j = c - P;
                for (int nn = -P; nn <= P; ++nn) a = cmac(a, tb[nn - j + 2 * P], src[nn + P]);
            }
            acc[c] = a;
        }
    }
    __syncthreads();
    cd* o = loc + (int64_t)rhs * A.ncoef + A.eoff[b];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) o[c] = acc[c];
}

// Helmholtz M2L split into chunks of List-2 entries: one CTA per chunk, thread
// (c, s) owns output c for source lane s; the S lanes' sums are combined in a
// fixed order into one partial sum per chunk, and k_m2l_reduce adds the chunks
// of a box in chunk order (bitwise reproducible, and the long all-pairs lists
// of the top level are spread over many CTAs).
constexpr int kM2LChunk = 32;

__global__ void k_m2l_chunk(M2LArgs A, int ch0, const int* __restrict__ chunk_box, const int* __restrict__ cq0,
                            const int* __restrict__ cq1, int P, int S, cd* __restrict__ part, int64_t part_stride,
                            const cd* __restrict__ mp) {
    extern __shared__ cd sm[];
    int ch = ch0 + blockIdx.x;
    int rhs = blockIdx.y;
    int b = chunk_box[ch];
    int l = A.blevel[b];
    int nc = 2 * P + 1, nt = 4 * P + 1;
    int t = threadIdx.x;
    int c = t % nc, sl = t / nc;
    bool act = sl < S;
    cd* msrc = sm;                         // [S][nc]
    cd* mtab = sm + (size_t)S * nc;        // [S][nt]
    cd acc = {0, 0};
    int q0 = cq0[ch], q1 = cq1[ch];
    for (int qb = q0; qb < q1; qb += S) {
        __syncthreads();
        int nsrc = min(S, q1 - qb);
        for (int i = t; i < nsrc * nc; i += blockDim.x) {
            int ss = i / nc, cc = i - ss * nc;
            int src = A.lent[qb + ss];
            msrc[(size_t)ss * nc + cc] = mp[(int64_t)rhs * A.ncoef + A.eoff[src] + cc];
        }
        for (int i = t; i < nsrc * nt; i += blockDim.x) {
            int ss = i / nt, cc = i - ss * nt;
            int q = qb + ss;
            mtab[(size_t)ss * nt + cc] = A.tab[A.tbase[l] + (int64_t)(q - A.tq0[l]) * nt + cc];
        }
        __syncthreads();
        if (act && sl < nsrc) {
            const cd* ms = msrc + (size_t)sl * nc;
            const cd* tb = mtab + (size_t)sl * nt + (nc - 1 - c);   // T[n - c + 2P] = tb[n]
            cd a = acc;
            for (int nn = 0; nn < nc; ++nn) a = cmac(a, tb[nn], ms[nn]);
            acc = a;
        }
    }
    __syncthreads();
    cd* red = sm;                          // [S][nc]
    if (act) red[(size_t)sl * nc + c] = acc;
    __syncthreads();
    if (t < nc) {
        cd v = red[t];
        for (int ss = 1; ss < S; ++ss) v += red[(size_t)ss * nc + t];
        part[(int64_t)rhs * part_stride + (int64_t)(ch - ch0) * nc + t] = v;
    }
}

__global__ void k_m2l_reduce(int lo, int nbl, const int* __restrict__ box_chunk0, int ch0, int nc,
                             const cd* __restrict__ part, int64_t part_stride, const int64_t* __restrict__ eoff,
                             int64_t ncoef, cd* __restrict__ loc) {
    int b = lo + blockIdx.x;
    int rhs = blockIdx.y;
    int c0 = box_chunk0[b], c1 = box_chunk0[b + 1];
    cd* out = loc + (int64_t)rhs * ncoef + eoff[b];
    const cd* pp = part + (int64_t)rhs * part_stride;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        cd v = {0, 0};
        for (int k = c0; k < c1; ++k) v += pp[(int64_t)(k - ch0) * nc + c];
        out[c] = v;
    }
}

// ---------------------------------------------------------------------------
// M2P (step 5, List 3) and L2P (step 8): one CTA per leaf, one thread per target
// ---------------------------------------------------------------------------
template <int KER>
__global__ void k_eval(ExpArgs A, const int* __restrict__ leaves, const int* __restrict__ l3off,
                       const int* __restrict__ l3, const cd* __restrict__ mp, const cd* __restrict__ loc,
                       cd* __restrict__ u, int maxP, const cd* __restrict__ lrow, int RL, int do_l2p) {
    extern __shared__ cd sm[];
    int b = leaves[blockIdx.x];
    int rhs = blockIdx.y;
    int P = A.Plev[A.blevel[b]];
    int nc = 2 * P + 1;
    cd* coef = sm;                                  // 2*maxP+1
    cd* rows = sm + 2 * maxP + 1;                   // per thread: maxP+2 (Helmholtz L2P)
    int s0 = A.bst[b], s1 = A.ben[b];
    for (int t0 = s0; t0 < s1; t0 += blockDim.x) {
        int i = t0 + threadIdx.x;
        bool valid = i < s1;
        cd x0 = {0, 0}, x1 = {0, 0};
        if (valid) {
            x0 = cd{A.xr[i], A.xi[i]};
            x1 = cd{A.xr[A.n + i], A.xi[A.n + i]};
        }
        cd acc = {0, 0};
        // M2P over List 3
        for (int q = l3off[b]; q < l3off[b + 1]; ++q) {
            int s = l3[q];
            int Ps = A.Plev[A.blevel[s]];
            int ns = 2 * Ps + 1;
            __syncthreads();
            const cd* m = mp + (int64_t)rhs * A.ncoef + A.eoff[s];
            for (int c = threadIdx.x; c < ns; c += blockDim.x) coef[c] = m[c];
            __syncthreads();
            if (!valid) continue;
            cd z, e;
            zeta_eta(x0 - cd{A.cre[2 * s], A.cim[2 * s]}, x1 - cd{A.cre[2 * s + 1], A.cim[2 * s + 1]}, z, e);
            if (KER == CFMM_LAPLACE) {
                acc += (0.5 * clog_p(z * e)) * coef[0];
                cd iz = cinv(z), ie = cinv(e), zp = iz, ep = ie;
                for (int nn = 1; nn <= Ps; ++nn) {
                    acc += coef[nn] * ep + coef[Ps + nn] * zp;
                    zp = zp * iz;
                    ep = ep * ie;
                }
            } else {
                // S_n(x - c) by forward recurrence in registers
                cd r = csqrt_p(z * e);
                cd zz = A.kappa * r;
                cd h0, h1;
                hankel01(zz, &h0, &h1);
                cd ir = cinv(r), uu = z * ir, vv = e * ir, zi = cinv(zz);
                acc += coef[Ps] * h0;
                cd hm = h0, hn = h1, up = uu, vp = vv;
                for (int nn = 1; nn <= Ps; ++nn) {
                    cd neg = (nn & 1) ? -hn : hn;
                    acc = cmac(cmac(acc, coef[Ps + nn], hn * up), coef[Ps - nn], neg * vp);
                    cd hp = rmac(-hm, 2.0 * nn, zi * hn);
                    hm = hn;
                    hn = hp;
                    up = up * uu;
                    vp = vp * vv;
                }
            }
        }
        if (!do_l2p) {
            // M2P only (the L2P runs in complex64): leaves without List 3 add nothing
            if (valid && l3off[b + 1] > l3off[b]) u[(int64_t)rhs * A.n + i] += acc;
            continue;
        }
        // L2P
        __syncthreads();
        const cd* lc = loc + (int64_t)rhs * A.ncoef + A.eoff[b];
        for (int c = threadIdx.x; c < nc; c += blockDim.x) coef[c] = lc[c];
        __syncthreads();
        if (valid) {
            cd z, e;
            zeta_eta(x0 - cd{A.cre[2 * b], A.cim[2 * b]}, x1 - cd{A.cre[2 * b + 1], A.cim[2 * b + 1]}, z, e);
            if (KER == CFMM_LAPLACE) {
                acc += coef[0];
                cd zp = z, ep = e;
                for (int nn = 1; nn <= P; ++nn) {
                    acc += coef[nn] * zp + coef[P + nn] * ep;
                    zp = zp * z;
                    ep = ep * e;
                }
            } else if (lrow) {
                // T_k(x - c) = (-1)^k T_k(c - x), the plan's row of this point
                const cd* t = lrow + (int64_t)i * RL + (P + 1);
                acc += coef[P] * t[0];
                for (int nn = 1; nn <= P; ++nn) {
                    cd tp = t[nn], tm = t[-nn];
                    if (nn & 1) {
                        tp = -tp;
                        tm = -tm;
                    }
                    acc = cmac(cmac(acc, coef[P + nn], tp), coef[P - nn], tm);
                }
            } else {
                cd* row = rows + (size_t)threadIdx.x * (maxP + 2);
                cd r = csqrt_p(z * e);
                if (r.x == 0.0 && r.y == 0.0) {
                    acc += coef[P];
                } else {
                    bessel_j_seq(A.kappa * r, P, row);
                    cd ir = cinv(r), uu = z * ir, vv = e * ir, up = uu, vp = vv;
                    acc += coef[P] * row[0];
                    for (int nn = 1; nn <= P; ++nn) {
                        cd jn = row[nn];
                        cd neg = (nn & 1) ? -jn : jn;
                        acc += coef[P + nn] * (jn * up) + coef[P - nn] * (neg * vp);
                        up = up * uu;
                        vp = vp * vv;
                    }
                }
            }
            u[(int64_t)rhs * A.n + i] += acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Target gradients of M2P (List 3) and L2P (FP64), added to g [rhs][2][n]:
// d/dx1 = d/dzeta + d/deta, d/dx2 = i (d/dzeta - d/deta), with
//   Laplace  u = M0 log(zeta eta)/2 + sum Mp_n eta^-n + Mm_n zeta^-n:
//            d/dzeta = M0/(2 zeta) - sum n Mm_n zeta^-n-1 (likewise eta);
//            u = L0 + sum Lp_n zeta^n + Lm_n eta^n: d/dzeta = sum n Lp_n zeta^n-1;
//   Helmholtz d/dzeta T_n = (kappa/2) T_{n-1}, d/deta T_n = -(kappa/2) T_{n+1}
//            for T = S (M2P) and G (L2P).
// ---------------------------------------------------------------------------
template <int KER>
__global__ void k_eval_grad(ExpArgs A, const int* __restrict__ leaves, const int* __restrict__ l3off,
                            const int* __restrict__ l3, const cd* __restrict__ mp, const cd* __restrict__ loc,
                            cd* __restrict__ g, int maxP) {
    extern __shared__ cd sm[];
    int b = leaves[blockIdx.x];
    int rhs = blockIdx.y;
    int P = A.Plev[A.blevel[b]];
    cd* coef = sm;                                  // 2*maxP+1
    cd* rows = sm + 2 * maxP + 1;                   // per thread: 2*maxP+3 (Helmholtz rows n = -P-1..P+1)
    int s0 = A.bst[b], s1 = A.ben[b];
    const double kh = 0.5 * A.kappa;
    for (int t0 = s0; t0 < s1; t0 += blockDim.x) {
        int i = t0 + threadIdx.x;
        bool valid = i < s1;
        cd x0 = {0, 0}, x1 = {0, 0};
        if (valid) {
            x0 = cd{A.xr[i], A.xi[i]};
            x1 = cd{A.xr[A.n + i], A.xi[A.n + i]};
        }
        cd dz = {0, 0}, de = {0, 0};
        cd* row = rows + (size_t)threadIdx.x * (2 * maxP + 3);
        for (int q = l3off[b]; q < l3off[b + 1]; ++q) {
            int s = l3[q];
            int Ps = A.Plev[A.blevel[s]];
            __syncthreads();
            const cd* m = mp + (int64_t)rhs * A.ncoef + A.eoff[s];
            for (int c = threadIdx.x; c < 2 * Ps + 1; c += blockDim.x) coef[c] = m[c];
            __syncthreads();
            if (!valid) continue;
            cd z, e;
            zeta_eta(x0 - cd{A.cre[2 * s], A.cim[2 * s]}, x1 - cd{A.cre[2 * s + 1], A.cim[2 * s + 1]}, z, e);
            if (KER == CFMM_LAPLACE) {
                cd iz = cinv(z), ie = cinv(e);
                dz += 0.5 * (coef[0] * iz);
                de += 0.5 * (coef[0] * ie);
                cd zp = iz * iz, ep = ie * ie;   // zeta^-n-1
                for (int nn = 1; nn <= Ps; ++nn) {
                    dz -= (double)nn * (coef[Ps + nn] * zp);
                    de -= (double)nn * (coef[nn] * ep);
                    zp = zp * iz;
                    ep = ep * ie;
                }
            } else {
                cyl_row(1, z, e, A.kappa, Ps, row);          // S_n, n = -Ps-1..Ps+1
                for (int nn = -Ps; nn <= Ps; ++nn) {
                    cd c = coef[Ps + nn];
                    dz = cmac(dz, c, row[nn + Ps + 1 - 1]);
                    de = cmac(de, c, row[nn + Ps + 1 + 1]);
                }
            }
        }
        __syncthreads();
        const cd* lc = loc + (int64_t)rhs * A.ncoef + A.eoff[b];
        for (int c = threadIdx.x; c < 2 * P + 1; c += blockDim.x) coef[c] = lc[c];
        __syncthreads();
        if (!valid) continue;
        cd z, e;
        zeta_eta(x0 - cd{A.cre[2 * b], A.cim[2 * b]}, x1 - cd{A.cre[2 * b + 1], A.cim[2 * b + 1]}, z, e);
        cd lz = {0, 0}, le = {0, 0};
        if (KER == CFMM_LAPLACE) {
            cd zp = {1, 0}, ep = {1, 0};   // zeta^n-1
            for (int nn = 1; nn <= P; ++nn) {
                lz += (double)nn * (coef[nn] * zp);
                le += (double)nn * (coef[P + nn] * ep);
                zp = zp * z;
                ep = ep * e;
            }
        } else {
            cyl_row(0, z, e, A.kappa, P, row);               // G_n, n = -P-1..P+1
            for (int nn = -P; nn <= P; ++nn) {
                cd c = coef[P + nn];
                lz = cmac(lz, c, row[nn + P + 1 - 1]);
                le = cmac(le, c, row[nn + P + 1 + 1]);
            }
        }
        if (KER == CFMM_LAPLACE) {
            dz += lz;
            de += le;
        } else {
            dz = kh * (dz + lz);
            de = (-kh) * (de + le);
        }
        cd* go = g + (int64_t)rhs * 2 * A.n + i;
        go[0] += dz + de;
        go[A.n] += mul_i(dz - de);
    }
}

// ---------------------------------------------------------------------------
// L2P in complex64 arithmetic (mixed precision). With zeta~ = zeta/rho_b,
// eta~ = eta/rho_b (rho_b = sqrt(2)/2 w, the leaf's radius):
//   Laplace    u = L^_0 + sum L^_n zeta~^n + L^'_n eta~^n,  L^_n = L_n rho_b^n
//   Helmholtz  u = sum_n Jh_n(k r) (L^_n zeta~^n + L^_-n eta~^n),
//              L^_n = L_n (k rho_b/2)^n/n!,  L^_-n = (-1)^n L_-n (k rho_b/2)^n/n!
// (G_n = J_n(k r) (zeta/r)^n, G_-n = (-1)^n J_n(k r) (eta/r)^n), where
//   Jh_n(z) = J_n(z) n! (2/z)^n
// is entire in w = z^2 = (k rho_b)^2 zeta~ eta~ with Jh_n(0) = 1. From
// J_{n-1} + J_{n+1} = (2n/z) J_n,  Jh_{n-1} = Jh_n - (w/4) Jh_{n+1}/(n(n+1)),
// so the ratios q_n = Jh_n/Jh_{n-1} = 1/(1 - (w/4) q_{n+1}/(n(n+1))) follow by
// Miller's backward recurrence from q = 1, and Jh_0 = J_0 from
// exp(-+ i z) = J_0 + 2 sum (-+ i)^k J_k = Jh_0 (1 + 2 sum (-+ i z/2)^k/k! prod q).
// Coefficients are scaled in FP64 per leaf and rounded; the terms are added
// in a compensated (Kahan) FP32 sum.
// ---------------------------------------------------------------------------
constexpr int kL2p2fMaxP = 128;

template <int KER>
__global__ void __launch_bounds__(kExpThreads) k_l2p2f(ExpArgs A, const int* __restrict__ leaves,
                                                        const cd* __restrict__ loc, cd* __restrict__ u, double W) {
    extern __shared__ cf coef2[];
    int b = leaves[blockIdx.x];
    int rhs = blockIdx.y;
    int lev = A.blevel[b];
    int P = A.Plev[lev];
    int nc = 2 * P + 1;
    double rb = 0.70710678118654752440 * ldexp(W, -lev);
    const cd* lc = loc + (int64_t)rhs * A.ncoef + A.eoff[b];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        // Laplace layout [c0, zeta^1..zeta^P, eta^1..eta^P]; Helmholtz [c_-P .. c_P]
        int n = KER == CFMM_LAPLACE ? (c <= P ? c : c - P) : abs(c - P);
        double s = 1.0, g = KER == CFMM_LAPLACE ? rb : 0.5 * A.kappa * rb;
        for (int j = 1; j <= n; ++j) s *= KER == CFMM_LAPLACE ? g : g / j;
        if (KER != CFMM_LAPLACE && c < P && (n & 1)) s = -s;
        coef2[c] = to_cf(s * lc[c]);
    }
    __syncthreads();
    double irb = 1.0 / rb;
    cd c0 = {A.cre[2 * b], A.cim[2 * b]}, c1 = {A.cre[2 * b + 1], A.cim[2 * b + 1]};
    cf G[kL2p2fMaxP + 1];
    for (int i = A.bst[b] + threadIdx.x; i < A.ben[b]; i += blockDim.x) {
        cd d0 = irb * (cd{A.xr[i], A.xi[i]} - c0), d1 = irb * (cd{A.xr[A.n + i], A.xi[A.n + i]} - c1);
        cf zt = to_cf(d0 + mul_i(d1)), et = to_cf(d0 - mul_i(d1));
        Kahan acc;
        if (KER == CFMM_LAPLACE) {
            acc.add(coef2[0]);
            cf zp = zt, ep = et;
            for (int nn = 1; nn <= P; ++nn) {
                acc.add(cmacf(coef2[nn] * zp, coef2[P + nn], ep));
                zp = zp * zt;
                ep = ep * et;
            }
        } else {
            float kr = (float)(A.kappa * rb);
            cf w = (kr * kr) * (zt * et);
            cf zz = csqrtf_p(w);
            float big = fmaxf((float)P, hypotf(zz.x, zz.y));
            int N = (int)big + 12 + (int)sqrtf(8.f * big);
            bool up = zz.y >= 0.f;
            cf a = 0.5f * (up ? cf{zz.y, -zz.x} : cf{-zz.y, zz.x});   // -+ i z / 2
            cf q = {1.f, 0.f}, H = {1.f, 0.f};
            for (int nn = N; nn >= 1; --nn) {
                float den = 0.25f / ((float)nn * (float)(nn + 1));
                q = cinvf(cf{1.f, 0.f} - (den * w) * q);
                if (nn <= P) G[nn] = q;
                H = cf{1.f, 0.f} + (1.f / (float)nn) * (a * (q * H));
            }
            float ex = expf(2.f * a.x), sn, cs;
            sincosf(2.f * a.y, &sn, &cs);
            cf g = cf{ex * cs, ex * sn} * cinvf(2.f * H - cf{1.f, 0.f});
            acc.add(coef2[P] * g);
            cf zp = zt, ep = et;
            for (int nn = 1; nn <= P; ++nn) {
                g = g * G[nn];
                acc.add(g * cmacf(coef2[P + nn] * zp, coef2[P - nn], ep));
                zp = zp * zt;
                ep = ep * et;
            }
        }
        u[(int64_t)rhs * A.n + i] += acc.value();
    }
}

// table kernels (plan time)
__global__ void k_tab_m2l(int nq, const int* __restrict__ qbox, const int* __restrict__ lent,
                          const int* __restrict__ blevel, const int* __restrict__ Plev, const int64_t* __restrict__ tbase,
                          const int* __restrict__ tq0, const double* __restrict__ cre, const double* __restrict__ cim,
                          double kappa, cd* __restrict__ tab, int q_first) {
    int qi = blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= nq) return;
    int q = q_first + qi;
    int b = qbox[qi], s = lent[q];
    int l = blevel[b];
    int P = Plev[l];
    cd* t = tab + tbase[l] + (int64_t)(q - tq0[l]) * (4 * P + 1);
    // S_j(c_t - c_s), j = -2P..2P, stored at j + 2P
    cd z, e;
    zeta_eta(cd{cre[2 * b] - cre[2 * s], cim[2 * b] - cim[2 * s]},
             cd{cre[2 * b + 1] - cre[2 * s + 1], cim[2 * b + 1] - cim[2 * s + 1]}, z, e);
    cd r = csqrt_p(z * e);
    cd zz = kappa * r;
    cd h0, h1;
    hankel01(zz, &h0, &h1);
    cd ir = cinv(r), uu = z * ir, vv = e * ir, zi = cinv(zz);
    int M = 2 * P;
    t[M] = h0;
    cd hm = h0, hn = h1, up = uu, vp = vv;
    for (int j = 1; j <= M; ++j) {
        cd neg = (j & 1) ? -hn : hn;
        t[M + j] = hn * up;
        t[M - j] = neg * vp;
        cd hp = (2.0 * j) * (zi * hn) - hm;
        hm = hn;
        hn = hp;
        up = up * uu;
        vp = vp * vv;
    }
}

// per child box: G_j(c_parent - c_child), j = -(Pc+Pp)..(Pc+Pp); scratch row per thread
__global__ void k_tab_shift(int lo, int hi, const int* __restrict__ parent, const int* __restrict__ blevel,
                            const int* __restrict__ Plev, const int64_t* __restrict__ shoff,
                            const double* __restrict__ cre, const double* __restrict__ cim, double kappa,
                            cd* __restrict__ tab) {
    int b = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= hi) return;
    int p = parent[b];
    int Pc = Plev[blevel[b]], Pp = Plev[blevel[p]];
    int M = Pc + Pp;
    cd* t = tab + shoff[b];
    cd z, e;
    zeta_eta(cd{cre[2 * p] - cre[2 * b], cim[2 * p] - cim[2 * b]},
             cd{cre[2 * p + 1] - cre[2 * b + 1], cim[2 * p + 1] - cim[2 * b + 1]}, z, e);
    cd r = csqrt_p(z * e);
    // J_0..J_M into the positive half, then the angular factors
    bessel_j_seq(kappa * r, M, t + M);
    if (r.x == 0.0 && r.y == 0.0) {
        for (int j = 1; j <= M; ++j) t[M - j] = cd{0, 0};
        return;
    }
    cd ir = cinv(r), uu = z * ir, vv = e * ir, up = uu, vp = vv;
    for (int j = 1; j <= M; ++j) {
        cd f = t[M + j];
        cd neg = (j & 1) ? -f : f;
        t[M - j] = neg * vp;
        t[M + j] = f * up;
        up = up * uu;
        vp = vp * vv;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct PlanExt {
    cfmm_plan_s* P;
    Fmm2dState* S;
};
static std::mutex g_ext_mu;
static std::vector<PlanExt>& exts() {
    static std::vector<PlanExt> v;
    return v;
}

static Fmm2dState* state(cfmm_plan_s* P) {
    std::lock_guard<std::mutex> lk(g_ext_mu);
    for (auto& e : exts())
        if (e.P == P) return e.S;
    return nullptr;
}

void fmm2d_release(cfmm_plan_s* P) {
    std::lock_guard<std::mutex> lk(g_ext_mu);
    auto& v = exts();
    for (size_t i = 0; i < v.size(); ++i)
        if (v[i].P == P) {
            delete v[i].S;
            v.erase(v.begin() + i);
            return;
        }
}

// Sec. 6.3: expansion order per level (prefactors dropped, one digit of headroom)
static int nterms_laplace(int dim, int k, double eps) {
    double ratio = (std::sqrt((double)dim) * 0.5) / (k + 0.5);
    double t = 1.0;
    int n = 0;
    for (;;) {
        ++n;
        t *= ratio;
        if (t <= eps) return n;
    }
}

static int nterms_helm2d_upto(int k, double eps, double kappa, double w, int pmax) {
    double R = (k + 0.5) * w, r = std::sqrt(2.0) * 0.5 * w;
    std::vector<cd> J(pmax + 4), H(pmax + 4);
    bessel_j_seq(cd{kappa * r, 0.0}, pmax + 3, J.data());
    cd zR = {kappa * R, 0.0};
    hankel01(zR, &H[0], &H[1]);
    cd zi = cinv(zR);
    for (int m = 1; m < pmax + 3; ++m) H[m + 1] = (2.0 * m) * (zi * H[m]) - H[m - 1];
    std::vector<char> ok(pmax + 4);
    for (int m = 0; m < pmax + 4; ++m) {
        cd v = H[m] * J[m];
        double a = std::sqrt(cabs2(v));
        ok[m] = std::isfinite(a) && a <= eps;
    }
    for (int n = 1; n < pmax; ++n)
        if (ok[n] && ok[n + 1] && ok[n + 2] && ok[n + 3]) return n;
    return -1;
}

// smallest n with |H_n(kR) J_n(kr)| <= eps for n..n+3 (search up to 2000; a
// short search range first, since the answer is near k R for large k R and
// O(log eps) otherwise)
static int nterms_helm2d(int k, double eps, double kappa, double w) {
    int guess = (int)(kappa * (k + 0.5) * w) + 80;
    if (guess < 2000) {
        int n = nterms_helm2d_upto(k, eps, kappa, w, guess);
        if (n > 0) return n;
    }
    int n = nterms_helm2d_upto(k, eps, kappa, w, 2000);
    return n > 0 ? n : 2000;
}

// the criterion is applied at eps * headroom: one digit for Laplace, two for
// Helmholtz (|H_n(kR) J_n(kr)| carries an extra 1/(n pi) against (r/R)^n)
constexpr double kPHeadroom = 0.1;
constexpr double kPHeadroomHelm = 0.01;

// First part of the setup, run before the lists are built: orders, offsets,
// the leaves and (Helmholtz) the per-point row table, launched on the side
// stream so that it overlaps the construction of the lists.
void fmm2d_presetup(cfmm_plan_s* P) {
    TreeDev& T = P->tree;
    cudaStream_t st = P->stream;
    PhaseTimer pt(st);
    Fmm2dState* S = new Fmm2dState();
    {
        std::lock_guard<std::mutex> lk(g_ext_mu);
        exts().push_back(PlanExt{P, S});
    }
    S->ker = P->kernel;
    S->l0 = T.l0;
    S->nlev = T.nlevels;
    S->Plev.assign(T.nlevels, 0);
    for (int l = 0; l < T.nlevels; ++l) {
        if (P->kernel == CFMM_LAPLACE) S->Plev[l] = nterms_laplace(2, P->sep, P->eps * kPHeadroom);
        // Helmholtz levels above the top expansion level carry no expansions:
        // their (large, host-evaluated) orders are not computed and read 0
        else if (l >= S->l0 || T.nboxes <= 1)
            S->Plev[l] = nterms_helm2d(P->sep, P->eps * kPHeadroomHelm, P->kappa, std::ldexp(P->W, -l));
    }
    P->P = S->Plev;
    pt.mark("setup:orders");
    if (T.nboxes <= 1) return;   // single leaf: near field only
    int maxP = 0;
    for (int l = S->l0; l < T.nlevels; ++l) maxP = std::max(maxP, S->Plev[l]);
    CFMM_REQUIRE(maxP <= 1000, CFMM_EUNSUPPORTED, "expansion order above 1000 at the top expansion level");
    S->maxP = maxP;
    P->maxP = maxP;
    S->dPlev.alloc(T.nlevels);
    upload(S->dPlev.get(), S->Plev.data(), sizeof(int) * T.nlevels, st);
    // coefficient offsets
    std::vector<int64_t> off(T.nboxes, -1);
    int64_t tot = 0;
    for (int l = S->l0; l < T.nlevels; ++l)
        for (int b = T.level_off[l]; b < T.level_off[l + 1]; ++b) {
            off[b] = tot;
            tot += 2 * S->Plev[l] + 1;
        }
    S->ncoef = tot;
    P->ncoef = tot;
    S->exp_off.alloc(T.nboxes);
    upload(S->exp_off.get(), off.data(), sizeof(int64_t) * T.nboxes, st);
    // leaves at level >= l0 (all leaves when the tree has more than one box);
    // boxes are level-major, so a box's level follows from the level offsets
    auto level_of = [&](int b) {
        return (int)(std::upper_bound(T.level_off.begin(), T.level_off.end(), b) - T.level_off.begin()) - 1;
    };
    S->maxP_leaf = 0;
    int lmin = T.nlevels;
    for (int b : T.leaf_boxes) {
        int lb = level_of(b);
        if (lb >= S->l0) {
            S->leaves_l0.push_back(b);
            S->maxP_leaf = std::max(S->maxP_leaf, S->Plev[lb]);
            lmin = std::min(lmin, lb);
        }
    }
    // a leaf's List 3 boxes lie below its level: their orders and the leaf's
    // own are at most the largest order at or below the coarsest leaf level
    S->maxP_fine = 0;
    for (int l = lmin; l < T.nlevels; ++l) S->maxP_fine = std::max(S->maxP_fine, S->Plev[l]);
    S->d_leaves_l0.alloc(S->leaves_l0.size());
    upload(S->d_leaves_l0.get(), S->leaves_l0.data(), sizeof(int) * S->leaves_l0.size(), st);
    pt.mark("setup:leaves");
    if (P->kernel == CFMM_HELMHOLTZ && !S->leaves_l0.empty()) {
        // on the side stream, beside the lists and the translation tables
        S->RL = 2 * S->maxP_leaf + 3;
        S->lrow.alloc((size_t)P->n * S->RL);
        S->rows_side = true;
        k_leaf_rows<<<(unsigned)S->leaves_l0.size(), 64, 0, near_fork(P)>>>(
            S->d_leaves_l0.get(), T.level.get(), T.start.get(), T.end.get(), S->dPlev.get(), P->xr.get(),
            P->xi.get(), P->n, T.cen_re.get(), T.cen_im.get(), P->kappa, S->RL, S->lrow.get());
        CFMM_LAUNCHED();
    }
}

// The rest of the setup, once the lists exist: P2L boxes, translation tables,
// List-2 chunks; joins the side stream's row table at the end.
void fmm2d_setup(cfmm_plan_s* P) {
    TreeDev& T = P->tree;
    cudaStream_t st = P->stream;
    if (!state(P)) fmm2d_presetup(P);
    Fmm2dState* S = state(P);
    PhaseTimer pt(st);
    if (T.nboxes <= 1) return;   // single leaf: near field only
    int maxP = S->maxP;
    // boxes that receive P2L contributions
    {
        const std::vector<int>& l4 = T.hloff[3];
        std::vector<int> boxes;
        for (int b = T.level_off[S->l0]; b < T.nboxes; ++b)
            if (l4[b + 1] > l4[b]) boxes.push_back(b);
        S->n_p2l = (int)boxes.size();
        S->d_p2l_boxes.alloc(boxes.size());
        if (!boxes.empty())
            upload(S->d_p2l_boxes.get(), boxes.data(), sizeof(int) * boxes.size(), st);
    }
    pt.mark("setup:p2l");
    // binomials C(n, k), n, k <= 2 maxP + 1 (exact integers up to 2^53, then rounded)
    S->NB = 2 * maxP + 2;
    {
        int NB = S->NB;
        std::vector<double> bt((size_t)(NB + 1) * (NB + 1), 0.0);
        for (int n = 0; n <= NB; ++n) {
            bt[(size_t)n * (NB + 1)] = 1.0;
            for (int k = 1; k <= n; ++k)
                bt[(size_t)n * (NB + 1) + k] = bt[(size_t)(n - 1) * (NB + 1) + k - 1] + (k <= n - 1 ? bt[(size_t)(n - 1) * (NB + 1) + k] : 0.0);
        }
        S->binom.alloc(bt.size());
        // (a copy from pageable memory returns once the source is staged)
        upload(S->binom.get(), bt.data(), sizeof(double) * bt.size(), st);
    }
    if (P->kernel == CFMM_HELMHOLTZ) {
        // M2L tables, level-major like List 2 itself
        const std::vector<int>& loff = T.hloff[1];
        S->m2l_base.assign(T.nlevels, 0);
        S->m2l_q0.assign(T.nlevels, 0);
        int64_t base = 0;
        for (int l = 0; l < T.nlevels; ++l) {
            int q0 = loff[T.level_off[l]], q1 = loff[T.level_off[l + 1]];
            S->m2l_base[l] = base;
            S->m2l_q0[l] = q0;
            if (l >= S->l0) base += (int64_t)(q1 - q0) * (4 * S->Plev[l] + 1);
        }
        S->t_m2l.alloc(base > 0 ? base : 1);
        S->d_m2l_base.alloc(T.nlevels);
        S->d_m2l_q0.alloc(T.nlevels);
        upload(S->d_m2l_base.get(), S->m2l_base.data(), sizeof(int64_t) * T.nlevels, st);
        upload(S->d_m2l_q0.get(), S->m2l_q0.data(), sizeof(int) * T.nlevels, st);
        // owner box of every List-2 entry at levels >= l0
        int qf = loff[T.level_off[S->l0]], ql = loff[T.nboxes];
        if (ql > qf) {
            std::vector<int> qbox(ql - qf);
            for (int b = T.level_off[S->l0]; b < T.nboxes; ++b)
                for (int q = loff[b]; q < loff[b + 1]; ++q) qbox[q - qf] = b;
            int* dq = plan_scratch().take_n<int>(qbox.size());
            upload(dq, qbox.data(), sizeof(int) * qbox.size(), st);
            int nq = ql - qf;
            // one warp per block: the few thousand pairs (one thread each) spread over
            // every SM instead of filling a fraction of them with larger blocks
            k_tab_m2l<<<(nq + 31) / 32, 32, 0, st>>>(nq, dq, T.lent[1].get(), T.level.get(), S->dPlev.get(),
                                                       S->d_m2l_base.get(), S->d_m2l_q0.get(), T.cen_re.get(),
                                                       T.cen_im.get(), P->kappa, S->t_m2l.get(), qf);
            CFMM_LAUNCHED();
        }
        pt.mark("setup:m2ltab");
        // List-2 chunks per box (levels >= l0)
        {
            std::vector<int> cb, c0v, c1v, bc0(T.nboxes + 1, 0);
            S->lvl_chunk0.assign(T.nlevels + 1, 0);
            S->lvl_part0.assign(T.nlevels + 1, 0);
            int64_t pslot = 0;
            for (int l = 0; l < T.nlevels; ++l) {
                S->lvl_chunk0[l] = (int)cb.size();
                S->lvl_part0[l] = pslot;
                // chunks of kM2LChunk entries (shorter chunks fill more SMs at a coarse
                // top level but spread each block's fixed per-coefficient work over
                // fewer sources: measured slower)
                int clen = kM2LChunk;
                for (int b = T.level_off[l]; b < T.level_off[l + 1]; ++b) {
                    bc0[b] = (int)cb.size();
                    if (l < S->l0) continue;
                    for (int q = loff[b]; q < loff[b + 1]; q += clen) {
                        cb.push_back(b);
                        c0v.push_back(q);
                        c1v.push_back(std::min(q + clen, loff[b + 1]));
                    }
                }
                if (l >= S->l0) pslot += (int64_t)((int)cb.size() - S->lvl_chunk0[l]) * (2 * S->Plev[l] + 1);
            }
            S->lvl_chunk0[T.nlevels] = (int)cb.size();
            S->lvl_part0[T.nlevels] = pslot;
            bc0[T.nboxes] = (int)cb.size();
            S->npart = pslot;
            S->chunk_box.alloc(cb.size());
            S->chunk_q0.alloc(cb.size());
            S->chunk_q1.alloc(cb.size());
            S->box_chunk0.alloc(T.nboxes + 1);
            if (!cb.empty()) {
                upload(S->chunk_box.get(), cb.data(), sizeof(int) * cb.size(), st);
                upload(S->chunk_q0.get(), c0v.data(), sizeof(int) * cb.size(), st);
                upload(S->chunk_q1.get(), c1v.data(), sizeof(int) * cb.size(), st);
            }
            upload(S->box_chunk0.get(), bc0.data(), sizeof(int) * (T.nboxes + 1), st);
        }
        pt.mark("setup:chunks");
        // shift tables for boxes at levels > l0
        std::vector<int64_t> so(T.nboxes, -1);
        int64_t sb = 0;
        for (int l = S->l0 + 1; l < T.nlevels; ++l)
            for (int b = T.level_off[l]; b < T.level_off[l + 1]; ++b) {
                so[b] = sb;
                sb += 2 * (S->Plev[l] + S->Plev[l - 1]) + 1;
            }
        S->t_shift.alloc(sb > 0 ? sb : 1);
        S->shift_off.alloc(T.nboxes);
        upload(S->shift_off.get(), so.data(), sizeof(int64_t) * T.nboxes, st);
        int lo = T.level_off[std::min(S->l0 + 1, T.nlevels)], hi = T.nboxes;
        if (hi > lo) {
            k_tab_shift<<<(hi - lo + 31) / 32, 32, 0, st>>>(lo, hi, T.parent.get(), T.level.get(), S->dPlev.get(),
                                                           S->shift_off.get(), T.cen_re.get(), T.cen_im.get(),
                                                           P->kappa, S->t_shift.get());
            CFMM_LAUNCHED();
        }
    }
    pt.mark("setup:shift");
    if (S->rows_side) near_join(P);
    pt.mark("setup:rowsjoin");
    for (auto f : {(const void*)k_point_to_exp<CFMM_LAPLACE>, (const void*)k_point_to_exp<CFMM_HELMHOLTZ>,
                   (const void*)k_m2m<CFMM_LAPLACE>, (const void*)k_m2m<CFMM_HELMHOLTZ>,
                   (const void*)k_l2l<CFMM_LAPLACE>, (const void*)k_l2l<CFMM_HELMHOLTZ>,
                   (const void*)k_m2l<CFMM_LAPLACE>, (const void*)k_m2l<CFMM_HELMHOLTZ>,
                   (const void*)k_m2l_chunk,
                   (const void*)k_eval<CFMM_LAPLACE>, (const void*)k_eval<CFMM_HELMHOLTZ>,
                   (const void*)k_eval_grad<CFMM_LAPLACE>, (const void*)k_eval_grad<CFMM_HELMHOLTZ>})
        CFMM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
}

template <int KER>
static void apply_t(cfmm_plan_s* P, Fmm2dState* S, const cd* sigma, const cd* tau, int64_t dstride, cd* u, int nrhs,
                    cd* g) {
    TreeDev& T = P->tree;
    cudaStream_t st = P->stream;
    auto rec = [&](int i) {
        if (P->timing) CFMM_CUDA(cudaEventRecord(P->ev[i], st));
    };
    KParams K{P->xr.get(), P->xi.get(), P->nr.get(), P->ni.get(), P->xr.get(), P->xi.get(), P->n, P->n,
              sigma, tau, dstride, P->slp, P->dlp, P->kappa};
    if (T.nboxes <= 1) {
        for (int i = 2; i <= 6; ++i) rec(i);
        launch_p2p(2, KER, K, T.d_leaf_boxes.get(), T.nleaves, T.start.get(), T.end.get(), T.loff[0].get(),
                   T.lent[0].get(), u, nrhs, false, st, P->precision == CFMM_MIXED);
        if (g)
            launch_p2p_grad(2, KER, K, T.d_leaf_boxes.get(), T.nleaves, T.start.get(), T.end.get(), T.loff[0].get(),
                            T.lent[0].get(), g, nrhs, st);
        rec(7);
        rec(8);
        return;
    }
    size_t need = (size_t)S->ncoef * nrhs;
    P->mpole.alloc(need);
    P->local.alloc(need);
    cd* mp = P->mpole.get();
    cd* lc = P->local.get();
    ExpArgs A{P->xr.get(), P->xi.get(), P->nr.get(), P->ni.get(), P->n, sigma, tau, dstride, P->slp, P->dlp,
              P->kappa, T.level.get(), T.start.get(), T.end.get(), T.cen_re.get(), T.cen_im.get(),
              S->dPlev.get(), S->exp_off.get(), S->ncoef};
    int maxP = S->maxP;
    // (3) P2P over List 1 (writes u) on the side stream, beside the far field
    {
        cudaStream_t ns = near_fork(P);
        launch_p2p(2, KER, K, S->d_leaves_l0.get(), (int)S->leaves_l0.size(), T.start.get(), T.end.get(),
                   T.loff[0].get(), T.lent[0].get(), u, nrhs, false, ns, P->precision == CFMM_MIXED);
        if (g)
            launch_p2p_grad(2, KER, K, S->d_leaves_l0.get(), (int)S->leaves_l0.size(), T.start.get(), T.end.get(),
                            T.loff[0].get(), T.lent[0].get(), g, nrhs, ns);
    }
    near_launched(P);
    // (1) P2M (shared memory sized by the leaves' orders)
    {
        int PL = S->maxP_leaf;
        int R = KER == CFMM_LAPLACE ? 2 * PL + 1 : 2 * PL + 3;
        int chunk = std::max(1, std::min(kExpThreads, (int)((96 * 1024) / ((R + 3) * sizeof(cd)))));
        size_t smem = sizeof(cd) * ((size_t)(2 * PL + 1) + (size_t)chunk * (R + 3));
        dim3 g((unsigned)S->leaves_l0.size(), nrhs);
        if (g.x) {
            k_point_to_exp<KER><<<g, kExpThreads, smem, st>>>(A, S->d_leaves_l0.get(), nullptr, nullptr, 0, mp, chunk,
                                                             S->lrow.get(), S->RL);
            CFMM_LAUNCHED();
        }
    }
    rec(2);
    // (2) M2M, finest level first
    TransArgs TA{T.level.get(), T.parent.get(), T.cbeg.get(), T.cend.get(), T.cen_re.get(), T.cen_im.get(),
                 S->dPlev.get(), S->exp_off.get(), S->ncoef, S->binom.get(), S->NB, S->t_shift.get(),
                 S->shift_off.get()};
    for (int l = T.nlevels - 2; l >= S->l0; --l) {
        int lo = T.level_off[l], nb = T.level_off[l + 1] - lo;
        int Pp = S->Plev[l], Pc = S->Plev[l + 1];
        size_t smem = sizeof(cd) * ((2 * Pp + 1) + (2 * Pc + 1) + 2 * (Pc + Pp) + 2);
        dim3 g(nb, nrhs);
        k_m2m<KER><<<g, kExpThreads, smem, st>>>(TA, lo, mp, mp, T.leaf.get());
        CFMM_LAUNCHED();
    }
    rec(3);
    // (4) M2L over List 2 (all levels >= l0)
    {
        M2LArgs MA{T.level.get(), T.cen_re.get(), T.cen_im.get(), S->dPlev.get(), S->exp_off.get(), S->ncoef,
                   T.loff[1].get(), T.lent[1].get(), S->binom.get(), S->NB, S->t_m2l.get(), S->d_m2l_base.get(),
                   S->d_m2l_q0.get()};
        int first = T.level_off[S->l0], nb = T.nboxes - first;
        if (KER == CFMM_HELMHOLTZ && maxP <= 255) {
            // chunks of List-2 entries, one launch per level (P fixed per level), then
            // the per-box reduction of the chunk sums
            P->m2l_part.alloc((size_t)S->npart * nrhs + 1);
            cd* part = P->m2l_part.get();
            for (int l = S->l0; l < T.nlevels; ++l) {
                int lo = T.level_off[l], nbl = T.level_off[l + 1] - lo;
                int ch0 = S->lvl_chunk0[l], nch = S->lvl_chunk0[l + 1] - ch0;
                if (nbl == 0) continue;
                int Pl = S->Plev[l], ncl = 2 * Pl + 1;
                cd* pl = part + S->lvl_part0[l];
                if (nch > 0) {
                    int Sl = std::max(1, std::min(8, 256 / ncl));
                    int threads = ((ncl * Sl + 31) / 32) * 32;
                    size_t smem = sizeof(cd) * (size_t)Sl * (ncl + 4 * Pl + 1);
                    dim3 gl(nch, nrhs);
                    k_m2l_chunk<<<gl, threads, smem, st>>>(MA, ch0, S->chunk_box.get(), S->chunk_q0.get(),
                                                            S->chunk_q1.get(), Pl, Sl, pl, S->npart, mp);
                    CFMM_LAUNCHED();
                }
                dim3 gr(nbl, nrhs);
                k_m2l_reduce<<<gr, 64, 0, st>>>(lo, nbl, S->box_chunk0.get(), ch0, ncl, pl, S->npart,
                                                S->exp_off.get(), S->ncoef, lc);
                CFMM_LAUNCHED();
            }
        } else {
            dim3 g(nb, nrhs);
            size_t smem = sizeof(cd) * (2 * (2 * maxP + 1) + 4 * maxP + 3);
            k_m2l<KER><<<g, 128, smem, st>>>(MA, first, mp, lc);
            CFMM_LAUNCHED();
        }
    }
    rec(4);
    // (6) P2L over List 4
    {
        int R = KER == CFMM_LAPLACE ? 2 * maxP + 1 : 2 * maxP + 3;
        int chunk = std::max(1, std::min(kExpThreads, (int)((96 * 1024) / ((R + 3) * sizeof(cd)))));
        size_t smem = sizeof(cd) * ((size_t)(2 * maxP + 1) + (size_t)chunk * (R + 3));
        if (S->n_p2l > 0) {
            dim3 g(S->n_p2l, nrhs);
            k_point_to_exp<KER><<<g, kExpThreads, smem, st>>>(A, S->d_p2l_boxes.get(), T.loff[3].get(),
                                                             T.lent[3].get(), 1, lc, chunk, nullptr, 0);
            CFMM_LAUNCHED();
        }
    }
    rec(5);
    // (7) L2L, coarsest level first
    for (int l = S->l0 + 1; l < T.nlevels; ++l) {
        int lo = T.level_off[l], nb = T.level_off[l + 1] - lo;
        int Pp = S->Plev[l - 1], Pc = S->Plev[l];
        size_t smem = sizeof(cd) * ((2 * Pp + 1) + 2 * (Pc + Pp) + 2);
        dim3 g(nb, nrhs);
        k_l2l<KER><<<g, kExpThreads, smem, st>>>(TA, lo, lc);
        CFMM_LAUNCHED();
    }
    rec(6);
    rec(7);
    near_join(P);   // the near field has written u
    // (5) M2P and (8) L2P (add to u; L2P in complex64 in mixed precision)
    {
        // with the plan's rows, L2P needs no per-thread row space
        size_t smem = sizeof(cd) * ((size_t)(2 * maxP + 1) + (S->lrow.get() ? 0 : (size_t)kExpThreads * (maxP + 2)));
        dim3 gr((unsigned)S->leaves_l0.size(), nrhs);
        bool l2p32 = P->precision == CFMM_MIXED && S->maxP_leaf <= kL2p2fMaxP;
        k_eval<KER><<<gr, kExpThreads, smem, st>>>(A, S->d_leaves_l0.get(), T.loff[2].get(), T.lent[2].get(), mp, lc,
                                                  u, maxP, S->lrow.get(), S->RL, l2p32 ? 0 : 1);
        CFMM_LAUNCHED();
        if (l2p32 && gr.x) {
            k_l2p2f<KER><<<gr, kExpThreads, sizeof(cf) * (2 * S->maxP_leaf + 1), st>>>(A, S->d_leaves_l0.get(), lc,
                                                                                        u, P->W);
            CFMM_LAUNCHED();
        }
        if (g && gr.x) {
            int Pg = S->maxP_fine;
            size_t gsm = sizeof(cd) * ((size_t)(2 * Pg + 1) + (size_t)kExpThreads * (2 * Pg + 3));
            CFMM_REQUIRE(gsm <= (size_t)kMaxSmem, CFMM_EUNSUPPORTED,
                         "2D gradient: leaf-level expansion order too large for the evaluation kernel");
            k_eval_grad<KER><<<gr, kExpThreads, gsm, st>>>(A, S->d_leaves_l0.get(), T.loff[2].get(), T.lent[2].get(),
                                                            mp, lc, g, Pg);
            CFMM_LAUNCHED();
        }
    }
    rec(8);
}

void fmm2d_apply(cfmm_plan_s* P, const cd* sigma, const cd* tau, int64_t dstride, cd* u, int nrhs, cd* g) {
    Fmm2dState* S = state(P);
    CFMM_REQUIRE(S, CFMM_EINVAL, "plan has no 2D state");
    if (P->kernel == CFMM_LAPLACE) apply_t<CFMM_LAPLACE>(P, S, sigma, tau, dstride, u, nrhs, g);
    else apply_t<CFMM_HELMHOLTZ>(P, S, sigma, tau, dstride, u, nrhs, g);
}

}  // namespace cfmm
