// 3D complex-coordinate Helmholtz FMM: expansions and translations (Sec. 5.3,
// Sec. 6.4), FP64.
//
// Expansion functions of a complex 3-vector x (x+ = x1 + i x2, x- = x1 - i x2,
// x3, rho^2 = x.x, rho the principal root; no angle is formed):
//   Z_n^m(x) = rho^n Y_n^m, Y the Schmidt semi-normalised harmonics of Sec. 3.2,
//     Z_0^0 = 1,  Z_m^m = -x+ sqrt((2m-1)/(2m)) Z_{m-1}^{m-1},  Z_{m+1}^m = sqrt(2m+1) x3 Z_m^m,
//     Z_n^m = A_n^m x3 Z_{n-1}^m - B_n^m rho^2 Z_{n-2}^m,
//     A_n^m = (2n-1)/sqrt((n-m)(n+m)),  B_n^m = sqrt((n-m-1)(n+m-1)/((n-m)(n+m))),
//     Z_n^{-m} = Z_n^m with x+ and x- exchanged;
//   R_n^m = j_n(k rho) rho^-n Z_n^m (entire),  S_n^m = h_n(k rho) rho^-n Z_n^m.
// Gegenbauer's addition theorem with Eq. sphaddition gives, for the
// constant-free kernel e^{ik r}/r = ik h_0(kr),
//   e^{ik|x-y|}/|x-y| = ik sum (2n+1) R_n^{-m}(y) S_n^m(x),
// hence (Thms 5.3.1, 5.3.2)
//   P2M  M_n^m = ik(2n+1) sum_j s_j R_n^{-m}(y_j - c)     M2P  u = sum M_n^m S_n^m(x - c)
//   P2L  L_n^m = ik(2n+1) sum_j s_j S_n^{-m}(y_j - c)     L2P  u = sum L_n^m R_n^m(x - c)
// and the double layer differentiates the source side along the normal:
//   grad(f_n rho^-n Z) = f_n rho^-n grad Z - k f_{n+1} rho^-(n+1) Z x,
//   n.grad Z_n^m = n3 c3 Z_{n-1}^m - nu+ s+ c+ Z_{n-1}^{m-1} + nu- s- c- Z_{n-1}^{m+1},
//   c3 = sqrt((n-m)(n+m)), c+ = sqrt((n+m)(n+m-1))/2, c- = sqrt((n-m)(n-m-1))/2,
//   s+ = 1 (m >= 1) else -1, s- = 1 (m >= 0) else -1, nu+- = n1 +- i n2.
//
// Translations by a complex shift d = c_new - c_old ("point and shoot",
// Sec. 5.3 translation operators):
//   1. rotate to the z-axis. e = (d1 + i d2)/s, s = sqrt(d1^2 + d2^2) (e = 1 if
//      s^2 = 0); t = sqrt(d.d); e_a = (d3 + i s)/t. The complex rotation
//      x' = R_y(a) R_z(-b) x carries d to (0, 0, t) and maps coefficients by
//        c' = Phi^-1 D^T E(e_a) D Phi E(e) c,   Phi = diag(i^m), E(e) = diag(e^m),
//      with D_n the real (2n+1)x(2n+1) matrix of the fixed rotation
//      x -> R_x(pi/2) x conjugated by Phi: the y-rotation of Eq. mp_y_rot
//      factored into two fixed rotations around a diagonal z-rotation.
//      D is built on the host by projecting onto the equator exactly as
//      Eq. mp_y_rot does (real rotation, so F_n is a trigonometric polynomial
//      and 2n+1 samples are exact);
//   2. re-expand along z with the exact coaxial coefficients
//        W_{n'}^m(x + t e3) = sum_n T^m_{n n'}(t) V_n^m(x)
//      (W = S, V = R for M2L, f = h; W = V = R or S, f = j for L2L and M2M),
//      generated per shift by the recurrences that follow from
//        d3 W_n^m = k(alpha_n^m W_{n-1}^m - beta_n^m W_{n+1}^m),
//        d- W_n^m = k(mu_n^m W_{n-1}^{m+1} + nu_n^m W_{n+1}^{m+1})  (m >= 0),
//        alpha = sqrt((n-m)(n+m))/(2n+1), beta = sqrt((n+1-m)(n+1+m))/(2n+1),
//        mu = sqrt((n-m)(n-m-1))/(2(2n+1)), nu = sqrt((n+m+1)(n+m+2))/(2(2n+1)):
//        T^0_{n,0} = (2n+1)(-1)^n f_n(kt),
//        T^m_{n,m} = [mu_{n+1}^{m-1} T^{m-1}_{n+1,m-1} + nu_{n-1}^{m-1} T^{m-1}_{n-1,m-1}] / nu_{m-1}^{m-1},
//        T_{n,n'+1} = [alpha_{n'} T_{n,n'-1} - alpha_{n+1} T_{n+1,n'} + beta_{n-1} T_{n-1,n'}] / beta_{n'},
//      the last only for n > n' (the stable direction); the rest from
//        T_{n',n} = (2n'+1)/(2n+1) (-1)^{n+n'} T_{n,n'},   T^{-m} = T^m.
//      These are the translations the paper's projection step approximates
//      (its Gauss-Legendre projection recovers T up to aliasing);
//   3. rotate back: c = E(1/e) Phi^-1 D^T E(1/e_a) D Phi c'.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>

#include "cfmm_special.cuh"
#include "kernels.cuh"

namespace cfmm {

namespace {

__host__ __device__ __forceinline__ int nmi(int n, int m) { return n * n + n + m; }

constexpr int kH3Threads = 256;
constexpr int kH3MaxP = kMaxP3Top;   // expansion order limit of this path
constexpr int kH3Smem = 220 * 1024;  // dynamic shared memory ceiling per block
constexpr int kM2LChunk3 = 32;       // List-2 entries per block when a list is split
constexpr int kTr3FlatMaxP = 23;     // largest order of the flat coaxial work
constexpr double kDegenTol = 1e-8;   // |d1^2 + d2^2| <= this * sum |d_i|^2: fixed-frame translation
constexpr int kTriMaxP = 40;         // largest M2L order whose coaxial operators are built ahead (k_tr3h_tri)
constexpr int kTriMaxPMulti = 56;    // the same with several right-hand sides (operators shared by all)
constexpr int kTriThreads = 128;     // threads of k_tr3h_tri
constexpr size_t kTriBudget = (size_t)6 << 30;   // bytes of operators per M2L launch range

// ---------------------------------------------------------------------------
// Per-device tables shared by all plans: D_n (row-major, n <= Pmax), the Z
// recurrence coefficients and the coaxial recurrence coefficients.
// ---------------------------------------------------------------------------
struct H3Tables {
    int Pmax = -1;
    DevBuf<double> Dh;       // D_n[m][m'] for m, m' >= 0, column-major per order
    DevBuf<int64_t> Dhoff;   // [Pmax+2]
    DevBuf<double> inv2n1;   // 1/(2n+1), n <= 2Pmax+2
    DevBuf<double> zA, zB;   // [(2Pmax+3)^2] by nmi(n, m), m >= 0
    DevBuf<double> al, be, ibe, mu, nu;  // coaxial recurrence coefficients, nmi(n, m), m >= 0
    DevBuf<double> g3, gp, gm;           // gradient coefficients c3, s+ c+, s- c- by nmi(n, m), all m
    DevBuf<double> dg, s21;  // sqrt((2m-1)/(2m)), sqrt(2m+1), m <= Pmax+1
    DevBuf<int> knm;         // k -> n * 256 + (m + 128), k < (Pmax+1)^2
    DevBuf<double> lsm, lsd; // eps_m s_n^m and eps_m / s_n^m, s = sqrt((n-|m|)! (n+|m|)!)
    DevBuf<double> fact, ifact;  // j! and 1/j!, j <= 2 Pmax + 2
    DevBuf<float> zAf, zBf, dgf, s21f;   // FP32 copies of zA, zB, dg, s21 (mixed-precision L2P)
};

// Tables only grow: a larger order builds a new set and the older sets stay
// alive, since plans that hold them may be running on other streams.
static std::mutex g_tab_mu;
static std::map<int, std::vector<H3Tables*>>& tab_map() {
    static std::map<int, std::vector<H3Tables*>> m;
    return m;
}

// Z_n^m at a complex point (host), n <= P, all m
static void host_ztable(int P, cd x0, cd x1, cd x2, std::vector<cd>& Z) {
    Z.assign((size_t)(P + 1) * (P + 1), cd{0, 0});
    cd xp = x0 + mul_i(x1), xm = x0 - mul_i(x1), z = x2;
    cd r2 = xp * xm + z * z;
    for (int sgn = 0; sgn < 2; ++sgn) {
        cd xs = sgn ? xm : xp;
        cd d = {1, 0};
        for (int m = 0; m <= P; ++m) {
            if (m > 0) d = (-std::sqrt((2.0 * m - 1.0) / (2.0 * m))) * (xs * d);
            if (sgn == 1 && m == 0) continue;
            int mi = sgn ? -m : m;
            Z[nmi(m, mi)] = d;
            if (m + 1 > P) continue;
            cd p2 = d, p1 = std::sqrt(2.0 * m + 1.0) * (z * d);
            Z[nmi(m + 1, mi)] = p1;
            for (int n = m + 2; n <= P; ++n) {
                double A = (2.0 * n - 1.0) / std::sqrt((double)(n - m) * (n + m));
                double B = std::sqrt((double)(n - m - 1) * (n + m - 1) / ((double)(n - m) * (n + m)));
                cd cur = A * (z * p1) - B * (r2 * p2);
                Z[nmi(n, mi)] = cur;
                p2 = p1;
                p1 = cur;
            }
        }
    }
}

// D_n for n <= P (real, row-major by (m + n, m' + n)); see the file comment.
static void host_rotation_tables(int P, std::vector<double>& D, std::vector<int64_t>& off) {
    const double kPi = 3.14159265358979323846;
    off.assign(P + 2, 0);
    for (int n = 0; n <= P; ++n) off[n + 1] = off[n] + (int64_t)(2 * n + 1) * (2 * n + 1);
    D.assign(off[P + 1], 0.0);
    std::vector<cd> Z, ab;
    // a_n^m = Y_n^m(e1), b_n^m = d_theta Y_n^m at (pi/2, 0) = -sqrt((n-m)(n+m)) Z_{n-1}^m(e1)
    host_ztable(P, cd{1, 0}, cd{0, 0}, cd{0, 0}, ab);
    std::vector<cd> F, G;
    for (int n = 0; n <= P; ++n) {
        int N = 2 * n + 1;
        // samples of Z_n^{m'} at p_j = X^T-rotated equator points and their
        // theta-derivative: frame x1 = Q x with Q = R_x(-pi/2)^T, so the
        // samples are taken at Q^T e_j = (cos phi, 0, -sin phi) along
        // Q^T (0, 0, -1) = (0, -1, 0) (v+ = -i, v- = i)
        F.assign((size_t)N * N, cd{0, 0});
        G.assign((size_t)N * N, cd{0, 0});
        for (int j = 0; j < N; ++j) {
            double ph = 2.0 * kPi * j / N;
            host_ztable(n, cd{std::cos(ph), 0}, cd{0, 0}, cd{-std::sin(ph), 0}, Z);
            for (int mp = -n; mp <= n; ++mp) {
                F[(size_t)j * N + (mp + n)] = Z[nmi(n, mp)];
                // grad Z . v = -i d+ Z + i d- Z
                cd g = {0, 0};
                if (n >= 1) {
                    if (std::abs(mp - 1) <= n - 1) {
                        double sp = mp >= 1 ? 1.0 : -1.0;
                        cd dp = (-0.5 * sp * std::sqrt((double)(n + mp) * (n + mp - 1))) * Z[nmi(n - 1, mp - 1)];
                        g = g - mul_i(dp);
                    }
                    if (std::abs(mp + 1) <= n - 1) {
                        double sm = mp >= 0 ? 1.0 : -1.0;
                        cd dm = (0.5 * sm * std::sqrt((double)(n - mp) * (n - mp - 1))) * Z[nmi(n - 1, mp + 1)];
                        g = g + mul_i(dm);
                    }
                }
                G[(size_t)j * N + (mp + n)] = g;
            }
        }
        for (int m = -n; m <= n; ++m) {
            double a = ab[nmi(n, m)].x;
            double b = 0.0;
            if (std::abs(m) <= n - 1) b = -std::sqrt((double)(n - m) * (n + m)) * ab[nmi(n - 1, m)].x;
            double den = a * a + b * b;
            for (int mp = -n; mp <= n; ++mp) {
                cd Fh = {0, 0}, Gh = {0, 0};
                for (int j = 0; j < N; ++j) {
                    double ph = 2.0 * kPi * j / N;
                    cd w = {std::cos(m * ph) / N, -std::sin(m * ph) / N};
                    Fh = Fh + w * F[(size_t)j * N + (mp + n)];
                    Gh = Gh + w * G[(size_t)j * N + (mp + n)];
                }
                cd da = (a * Fh + b * Gh) * (1.0 / den);
                // D = Phi DA Phi^-1: multiply by i^m i^-m'
                int e = ((m - mp) % 4 + 4) % 4;
                cd ph = e == 0 ? cd{1, 0} : e == 1 ? cd{0, 1} : e == 2 ? cd{-1, 0} : cd{0, -1};
                cd v = ph * da;
                CFMM_REQUIRE(std::fabs(v.y) <= 1e-10 * (1.0 + std::fabs(v.x)), CFMM_ECUDA,
                             "3D Helmholtz rotation table is not real");
                D[off[n] + (int64_t)(m + n) * N + (mp + n)] = v.x;
            }
        }
    }
}

static H3Tables* tables(int P) {
    int dev = 0;
    CFMM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tab_mu);
    auto& sets = tab_map()[dev];
    if (!sets.empty() && sets.back()->Pmax >= P) return sets.back();
    H3Tables* T = new H3Tables();
    int Pm = std::max(P, 16);
    std::vector<double> D;
    std::vector<int64_t> off;
    host_rotation_tables(Pm, D, off);
    int NN = 2 * Pm + 3;
    size_t NT = (size_t)NN * NN;
    std::vector<double> zA(NT, 0.0), zB(NT, 0.0), al(NT, 0.0), be(NT, 0.0), ibe(NT, 0.0), mu(NT, 0.0),
        nu(NT, 0.0), g3(NT, 0.0), gp(NT, 0.0), gm(NT, 0.0), dg(Pm + 2, 0.0), s21(Pm + 2, 0.0);
    for (int n = 0; n < NN; ++n) {
        for (int m = 0; m <= n; ++m) {
            int k = nmi(n, m);
            if (n >= m + 2) {
                zA[k] = (2.0 * n - 1.0) / std::sqrt((double)(n - m) * (n + m));
                zB[k] = std::sqrt((double)(n - m - 1) * (n + m - 1) / ((double)(n - m) * (n + m)));
            }
            al[k] = std::sqrt((double)(n - m) * (n + m)) / (2.0 * n + 1.0);
            be[k] = std::sqrt((double)(n + 1 - m) * (n + 1 + m)) / (2.0 * n + 1.0);
            ibe[k] = 1.0 / be[k];
            mu[k] = std::sqrt((double)(n - m) * std::max(n - m - 1, 0)) / (2.0 * (2.0 * n + 1.0));
            nu[k] = std::sqrt((double)(n + m + 1) * (n + m + 2)) / (2.0 * (2.0 * n + 1.0));
        }
        for (int m = -n; m <= n; ++m) {
            int k = nmi(n, m);
            g3[k] = std::sqrt((double)(n - m) * (n + m));
            gp[k] = (m >= 1 ? 0.5 : -0.5) * std::sqrt((double)(n + m) * std::max(n + m - 1, 0));
            gm[k] = (m >= 0 ? 0.5 : -0.5) * std::sqrt((double)(n - m) * std::max(n - m - 1, 0));
        }
    }
    for (int m = 1; m <= Pm + 1; ++m) dg[m] = std::sqrt((2.0 * m - 1.0) / (2.0 * m));
    for (int m = 0; m <= Pm + 1; ++m) s21[m] = std::sqrt(2.0 * m + 1.0);
    std::vector<int> knm((size_t)(Pm + 1) * (Pm + 1));
    for (int n = 0; n <= Pm; ++n)
        for (int m = -n; m <= n; ++m) knm[nmi(n, m)] = n * 256 + (m + 128);
    std::vector<int64_t> hoff(Pm + 2, 0);
    for (int n = 0; n <= Pm; ++n) hoff[n + 1] = hoff[n] + (int64_t)(n + 1) * (n + 1);
    std::vector<double> Dh(hoff[Pm + 1]);
    for (int n = 0; n <= Pm; ++n) {
        int N = 2 * n + 1;
        for (int m = 0; m <= n; ++m)
            for (int mp = 0; mp <= n; ++mp) Dh[hoff[n] + (int64_t)mp * (n + 1) + m] = D[off[n] + (int64_t)(m + n) * N + (mp + n)];
    }
    std::vector<double> inv2n1(NN);
    for (int n = 0; n < NN; ++n) inv2n1[n] = 1.0 / (2.0 * n + 1.0);
    auto up = [](DevBuf<double>& b, const std::vector<double>& v) {
        b.alloc(v.size());
        CFMM_CUDA(cudaMemcpy(b.get(), v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice));
    };
    up(T->Dh, Dh);
    up(T->inv2n1, inv2n1);
    T->Dhoff.alloc(hoff.size());
    CFMM_CUDA(cudaMemcpy(T->Dhoff.get(), hoff.data(), sizeof(int64_t) * hoff.size(), cudaMemcpyHostToDevice));
    up(T->mu, mu);
    up(T->nu, nu);
    up(T->g3, g3);
    up(T->gp, gp);
    up(T->gm, gm);
    up(T->dg, dg);
    up(T->s21, s21);
    {
        std::vector<double> f(2 * Pm + 3), fi(2 * Pm + 3), lm(knm.size()), ld(knm.size());
        f[0] = 1.0;
        for (int j = 1; j < (int)f.size(); ++j) f[j] = f[j - 1] * j;
        for (size_t j = 0; j < f.size(); ++j) fi[j] = 1.0 / f[j];
        for (int n = 0; n <= Pm; ++n)
            for (int m = -n; m <= n; ++m) {
                int am = std::abs(m);
                double sv = std::sqrt(f[n - am] * f[n + am]);
                double e = (m < 0 && (am & 1)) ? -1.0 : 1.0;
                lm[nmi(n, m)] = e * sv;
                ld[nmi(n, m)] = e / sv;
            }
        up(T->fact, f);
        up(T->ifact, fi);
        up(T->lsm, lm);
        up(T->lsd, ld);
    }
    T->knm.alloc(knm.size());
    CFMM_CUDA(cudaMemcpy(T->knm.get(), knm.data(), sizeof(int) * knm.size(), cudaMemcpyHostToDevice));
    {
        auto upf = [](DevBuf<float>& b, const std::vector<double>& v) {
            std::vector<float> f(v.begin(), v.end());
            b.alloc(f.size());
            CFMM_CUDA(cudaMemcpy(b.get(), f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice));
        };
        upf(T->zAf, zA);
        upf(T->zBf, zB);
        upf(T->dgf, dg);
        upf(T->s21f, s21);
    }

    T->zA.alloc(zA.size());
    T->zB.alloc(zB.size());
    T->al.alloc(al.size());
    T->be.alloc(be.size());
    T->ibe.alloc(ibe.size());

    CFMM_CUDA(cudaMemcpy(T->zA.get(), zA.data(), sizeof(double) * zA.size(), cudaMemcpyHostToDevice));
    CFMM_CUDA(cudaMemcpy(T->zB.get(), zB.data(), sizeof(double) * zB.size(), cudaMemcpyHostToDevice));
    CFMM_CUDA(cudaMemcpy(T->al.get(), al.data(), sizeof(double) * al.size(), cudaMemcpyHostToDevice));
    CFMM_CUDA(cudaMemcpy(T->be.get(), be.data(), sizeof(double) * be.size(), cudaMemcpyHostToDevice));
    CFMM_CUDA(cudaMemcpy(T->ibe.get(), ibe.data(), sizeof(double) * ibe.size(), cudaMemcpyHostToDevice));
    T->Pmax = Pm;
    sets.push_back(T);
    return T;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
struct ZCoef {
    const double* A;
    const double* B;
    const double* dg;    // sqrt((2m-1)/(2m))
    const double* s21;   // sqrt(2m+1)
    const int* knm;      // k -> n * 256 + (m + 128)
    const double* g3;    // gradient coefficients by nmi(n, m)
    const double* gp;
    const double* gm;
};

__device__ __forceinline__ void nm_tab(const int* knm, int k, int& n, int& m) {
    int v = __ldg(knm + k);
    n = v >> 8;
    m = (v & 255) - 128;
}

// Z table of (a0, a1, a2) up to order P into tab[nmi(n, m)]; columns split
// over threads t0, t0 + nthreads, ...
__device__ void z_table(ZCoef zc, cd a0, cd a1, cd a2, int P, cd* tab, int t0, int nthreads) {
    cd xp = a0 + mul_i(a1), xm = a0 - mul_i(a1), z = a2;
    cd r2 = xp * xm + z * z;
    for (int col = t0; col < 2 * P + 1; col += nthreads) {
        int m = col <= P ? col : col - P;
        bool neg = col > P;
        cd xs = neg ? xm : xp;
        cd d = {1, 0};
        for (int j = 1; j <= m; ++j) d = (-__ldg(zc.dg + j)) * (xs * d);
        int mi = neg ? -m : m;
        tab[nmi(m, mi)] = d;
        if (m + 1 > P) continue;
        cd p2 = d, p1 = __ldg(zc.s21 + m) * (z * d);
        tab[nmi(m + 1, mi)] = p1;
        for (int n = m + 2; n <= P; ++n) {
            int k = nmi(n, m);
            cd cur = zc.A[k] * (z * p1) - zc.B[k] * (r2 * p2);
            tab[nmi(n, mi)] = cur;
            p2 = p1;
            p1 = cur;
        }
    }
}

// F[n] = f_n(k rho) / rho^n for n = 0..N (f = j if reg, else h); rho = 0 (reg
// only) gives the limits k^n / (2n+1)!!
__device__ void radial_seq(bool reg, double kappa, cd r2, int N, cd* F) {
    cd rho = csqrt_p(r2);
    if (rho.x == 0.0 && rho.y == 0.0) {
        double v = 1.0;
        for (int n = 0; n <= N; ++n) {
            F[n] = cd{v, 0};
            v *= kappa / (2.0 * n + 3.0);
        }
        return;
    }
    cd z = kappa * rho;
    if (reg) sph_j_seq(z, N, F);
    else sph_h_seq(z, N, F);
    cd ir = cinv(rho), p = {1, 0};
    for (int n = 0; n <= N; ++n) {
        F[n] = F[n] * p;
        p = p * ir;
    }
}

__device__ __forceinline__ cd zget(const cd* tab, int n, int m) {
    if (n < 0 || m > n || -m > n) return cd{0, 0};
    return tab[nmi(n, m)];
}

struct Exp3hArgs {
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
    double kappa;
    ZCoef zc;
};

__device__ __forceinline__ void load3(const double* re, const double* im, int64_t n, int64_t j, cd* x) {
    for (int a = 0; a < 3; ++a) x[a] = cd{re[a * n + j], im[a * n + j]};
}

// P2M (sing = 0: R waves, the box's own points) or P2L (sing = 1: S waves,
// the box's List-4 leaves). Sources are staged chunk by chunk: Z table, radial
// factors and (sigma, tau, nu+, nu-, n3, y.n) per source; each thread owns
// coefficients and adds the sources' terms in source order.
__global__ void k_p2x3h(Exp3hArgs A, const int* __restrict__ boxes, const int* __restrict__ loff,
                        const int* __restrict__ lent, int sing, cd* __restrict__ out, int chunk) {
    extern __shared__ cd sm[];
    int b = boxes[blockIdx.x];
    int rhs = blockIdx.y;
    int P = A.Plev[A.blevel[b]];
    int nc = (P + 1) * (P + 1);
    cd* acc = sm;
    cd* tabs = acc + nc;                           // [chunk][nc]
    cd* rad = tabs + (size_t)chunk * nc;           // [chunk][P+2]
    cd* srcv = rad + (size_t)chunk * (P + 2);      // [chunk][6]
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
            int cols = 2 * P + 1;
            for (int w = threadIdx.x; w < cn * (cols + 1); w += blockDim.x) {
                int s = w / (cols + 1), col = w - s * (cols + 1);
                int64_t j = c0 + s;
                cd y[3];
                load3(A.xr, A.xi, A.n, j, y);
                for (int a = 0; a < 3; ++a) y[a] = y[a] - cen[a];
                if (col < cols) {
                    z_table(A.zc, y[0], y[1], y[2], P, tabs + (size_t)s * nc, col, cols);
                } else {
                    cd r2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
                    radial_seq(!sing, A.kappa, r2, P + 1, rad + (size_t)s * (P + 2));
                    cd* v = srcv + (size_t)s * 6;
                    v[0] = A.slp ? A.sigma[rhs * A.dstride + j] : cd{0, 0};
                    v[1] = A.dlp ? A.tau[rhs * A.dstride + j] : cd{0, 0};
                    if (A.dlp) {
                        cd nn[3];
                        load3(A.nr, A.ni, A.n, j, nn);
                        v[2] = nn[0] + mul_i(nn[1]);
                        v[3] = nn[0] - mul_i(nn[1]);
                        v[4] = nn[2];
                        v[5] = y[0] * nn[0] + y[1] * nn[1] + y[2] * nn[2];
                    }
                }
            }
            __syncthreads();
            for (int c = threadIdx.x; c < nc; c += blockDim.x) {
                int n, m;
                nm_tab(A.zc.knm, c, n, m);
                int mu = -m;
                cd a = acc[c];
                for (int s = 0; s < cn; ++s) {
                    const cd* tb = tabs + (size_t)s * nc;
                    const cd* F = rad + (size_t)s * (P + 2);
                    const cd* v = srcv + (size_t)s * 6;
                    cd Zv = tb[nmi(n, mu)];
                    cd term = {0, 0};
                    if (A.slp) term = v[0] * (F[n] * Zv);
                    if (A.dlp) {
                        cd g = {0, 0};
                        if (n >= 1) {
                            int kk = nmi(n, mu);
                            g = (__ldg(A.zc.g3 + kk) * v[4]) * zget(tb, n - 1, mu);
                            g = g - __ldg(A.zc.gp + kk) * (v[2] * zget(tb, n - 1, mu - 1));
                            g = g + __ldg(A.zc.gm + kk) * (v[3] * zget(tb, n - 1, mu + 1));
                        }
                        cd dw = F[n] * g - A.kappa * (F[n + 1] * (Zv * v[5]));
                        term += v[1] * dw;
                    }
                    a += term;
                }
                acc[c] = a;
            }
        }
    }
    __syncthreads();
    cd* o = out + (int64_t)rhs * A.ncoef + A.eoff[b];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        int n, m;
        nm_tab(A.zc.knm, c, n, m);
        cd v = mul_i(A.kappa * (2.0 * n + 1.0) * acc[c]);
        if (sing) o[c] += v;
        else o[c] = v;
    }
}

// Radial factors f_n(kappa rho)/rho^n, n <= P, of every point of the listed
// boxes relative to a box centre (one thread per point): the centre is the
// box itself (P2M, f = j) or, for P2L, the target box of List-4 entry q.
__global__ void k_radial3h(Exp3hArgs A, const int* __restrict__ boxes, int nboxes, const int* __restrict__ loff,
                           const int* __restrict__ lent, int sing, int P, const int* __restrict__ roff,
                           cd* __restrict__ rad) {
    int bi = blockIdx.x;
    if (bi >= nboxes) return;
    int b = boxes[bi];
    cd cen[3];
    for (int a = 0; a < 3; ++a) cen[a] = cd{A.cre[3 * b + a], A.cim[3 * b + a]};
    int qa = loff ? loff[b] : 0, qb = loff ? loff[b + 1] : 1;
    int64_t o = roff[bi];
    for (int q = qa; q < qb; ++q) {
        int src = loff ? lent[q] : b;
        int s0 = A.bst[src], s1 = A.ben[src];
        for (int j = s0 + threadIdx.x; j < s1; j += blockDim.x) {
            cd y[3];
            load3(A.xr, A.xi, A.n, j, y);
            for (int a = 0; a < 3; ++a) y[a] = y[a] - cen[a];
            radial_seq(!sing, A.kappa, y[0] * y[0] + y[1] * y[1] + y[2] * y[2], P,
                       rad + (o + (j - s0)) * (int64_t)(P + 1));
        }
        o += s1 - s0;
    }
}

// One harmonic column of a single-layer source: Z_n^{mu}(y) sigma for
// n = |mu|..P (mu >= 0 from x+, mu < 0 from x-, col = mu or P - mu), times
// the radial factor F[n] (Helmholtz; none for Laplace), added into acc at
// coefficient (n, -mu).
template <bool LAP>
__device__ __forceinline__ void p2x_column(const ZCoef& zc, int P, int col, cd xp, cd xm, cd z, cd r2, cd sg,
                                           const cd* __restrict__ F, cd* acc) {
    int am = col <= P ? col : col - P;
    bool neg = col > P;
    int m = neg ? am : -am;
    cd xs = neg ? xm : xp;
    cd d = sg;
    for (int i = 1; i <= am; ++i) d = (-__ldg(zc.dg + i)) * (xs * d);
    acc[nmi(am, m)] = LAP ? acc[nmi(am, m)] + d : cmac(acc[nmi(am, m)], F[am], d);
    if (am + 1 > P) return;
    cd p2 = d, p1 = __ldg(zc.s21 + am) * (z * d);
    acc[nmi(am + 1, m)] = LAP ? acc[nmi(am + 1, m)] + p1 : cmac(acc[nmi(am + 1, m)], F[am + 1], p1);
    for (int n = am + 2; n <= P; ++n) {
        int k = nmi(n, am);
        cd cur = __ldg(zc.A + k) * (z * p1) - __ldg(zc.B + k) * (r2 * p2);
        acc[nmi(n, m)] = LAP ? acc[nmi(n, m)] + cur : cmac(acc[nmi(n, m)], F[n], cur);
        p2 = p1;
        p1 = cur;
    }
}

// Single-layer P2M (sing = 0) / P2L (sing = 1). Each warp owns an accumulator
// row in shared memory and takes the (source, column) items of its box in
// rounds of 32 consecutive items, one per lane; with 2P+1 >= 32 columns the
// lanes of a round hold distinct columns, so they touch disjoint coefficients,
// and __syncwarp orders the rounds. With fewer columns a warp takes one source
// at a time, one lane per column. The warp rows are summed in warp order at
// the end, so the result does not depend on timing.
// LAP: the 3D Laplace P2M, M_n^m = (-1)^m sum sigma U_n^{-m}(y) with the
// regular solid harmonics U; since Z_n^{-m} = e s U_n^{-m} (s = sqrt((n-|m|)!
// (n+|m|)!), e = +-1 as in lsd), M_n^m = lsd_n^m sum sigma Z_n^{-m}(y).
template <bool LAP>
__global__ void k_p2x3h_slp(Exp3hArgs A, const int* __restrict__ boxes, const int* __restrict__ loff,
                            const int* __restrict__ lent, int sing, const int* __restrict__ roff,
                            const cd* __restrict__ rad, cd* __restrict__ out, const double* __restrict__ lsd) {
    extern __shared__ cd sm[];
    int bi = blockIdx.x;
    int b = boxes[bi];
    int rhs = blockIdx.y;
    int P = A.Plev[A.blevel[b]];
    int nc = (P + 1) * (P + 1);
    int C = 2 * P + 1;
    int nwarp = blockDim.x >> 5, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    cd* accw = sm + (size_t)wid * nc;
    for (int c = lane; c < nc; c += 32) accw[c] = cd{0, 0};
    __syncwarp();
    cd cen[3];
    for (int a = 0; a < 3; ++a) cen[a] = cd{A.cre[3 * b + a], A.cim[3 * b + a]};
    int qa = loff ? loff[b] : 0, qb = loff ? loff[b + 1] : 1;
    int64_t o = roff ? roff[bi] : 0;
    for (int q = qa; q < qb; ++q) {
        int src = loff ? lent[q] : b;
        int s0 = A.bst[src], s1 = A.ben[src];
        if (C >= 32) {
            int items = (s1 - s0) * C;
            for (int base = wid * 32; base < items; base += nwarp * 32) {
                int it = base + lane;
                if (it < items) {
                    int js = it / C, col = it - js * C;
                    int j = s0 + js;
                    cd y[3];
                    load3(A.xr, A.xi, A.n, j, y);
                    for (int a = 0; a < 3; ++a) y[a] = y[a] - cen[a];
                    cd xp = y[0] + mul_i(y[1]), xm = y[0] - mul_i(y[1]), z = y[2];
                    p2x_column<LAP>(A.zc, P, col, xp, xm, z, xp * xm + z * z, A.sigma[rhs * A.dstride + j],
                                    LAP ? nullptr : rad + (o + js) * (int64_t)(P + 1), accw);
                }
                __syncwarp();
            }
        } else {
            for (int j = s0 + wid; j < s1; j += nwarp) {
                if (lane < C) {
                    cd y[3];
                    load3(A.xr, A.xi, A.n, j, y);
                    for (int a = 0; a < 3; ++a) y[a] = y[a] - cen[a];
                    cd xp = y[0] + mul_i(y[1]), xm = y[0] - mul_i(y[1]), z = y[2];
                    p2x_column<LAP>(A.zc, P, lane, xp, xm, z, xp * xm + z * z, A.sigma[rhs * A.dstride + j],
                                    LAP ? nullptr : rad + (o + (j - s0)) * (int64_t)(P + 1), accw);
                }
            }
        }
        o += s1 - s0;
    }
    __syncthreads();
    cd* op = out + (int64_t)rhs * A.ncoef + A.eoff[b];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        cd v = {0, 0};
        for (int w = 0; w < nwarp; ++w) v += sm[(size_t)w * nc + c];
        if (LAP) {
            v = __ldg(lsd + c) * v;
        } else {
            int n, m;
            nm_tab(A.zc.knm, c, n, m);
            v = mul_i(A.kappa * (2.0 * n + 1.0) * v);
        }
        if (sing) op[c] += v;
        else op[c] = v;
    }
}

// Sum over n, m of coef_n^m F[n] Z_n^m(x) with Z generated column by column.
__device__ cd eval_wave(ZCoef zc, cd a0, cd a1, cd a2, int P, const cd* F, const cd* coef) {
    cd xp = a0 + mul_i(a1), xm = a0 - mul_i(a1), z = a2;
    cd r2 = xp * xm + z * z;
    cd acc = {0, 0};
    for (int sgn = 0; sgn < 2; ++sgn) {
        cd xs = sgn ? xm : xp;
        cd d = {1, 0};
        for (int m = 0; m <= P; ++m) {
            if (m > 0) d = (-__ldg(zc.dg + m)) * (xs * d);
            if (sgn == 1 && m == 0) continue;
            int mi = sgn ? -m : m;
            acc = cmac(acc, F[m], d * coef[nmi(m, mi)]);
            if (m + 1 > P) continue;
            cd p2 = d, p1 = __ldg(zc.s21 + m) * (z * d);
            acc = cmac(acc, F[m + 1], p1 * coef[nmi(m + 1, mi)]);
            for (int n = m + 2; n <= P; ++n) {
                int k = nmi(n, m);
                cd cur = zc.A[k] * (z * p1) - zc.B[k] * (r2 * p2);
                acc = cmac(acc, F[n], cur * coef[nmi(n, mi)]);
                p2 = p1;
                p1 = cur;
            }
        }
    }
    return acc;
}

// Target gradient of sum c_n^m F_n Z_n^m (F_n = f_n(k rho)/rho^n, f = j or h):
// grad(F_n Z) = F_n grad Z - k F_{n+1} Z x with dz Z_n^m = g3 Z_{n-1}^m,
// d+ Z_n^m = -gp Z_{n-1}^{m-1}, d- Z_n^m = gm Z_{n-1}^{m+1} (the tables g3, gp,
// gm of the double layer), so in one pass over Z_{n'}^{m'}, n' <= P (F given
// for n <= P + 1):
//   Dz = sum g3(n'+1, m') c_{n'+1}^{m'} F_{n'+1} Z,  D+ = sum -gp(n'+1, m'+1)
//   c_{n'+1}^{m'+1} F_{n'+1} Z,  D- = sum gm(n'+1, m'-1) c_{n'+1}^{m'-1} F_{n'+1} Z,
//   B = sum c_{n'}^{m'} F_{n'+1} Z;
// grad = (D+ + D- - k x1 B, i (D+ - D-) - k x2 B, Dz - k x3 B).
__device__ void eval_wave_grad(ZCoef zc, cd a0, cd a1, cd a2, int P, const cd* F, const cd* coef, cd& Dz, cd& Dp,
                               cd& Dm, cd& B) {
    cd xp = a0 + mul_i(a1), xm = a0 - mul_i(a1), z = a2;
    cd r2 = xp * xm + z * z;
    auto c = [&](int n, int m) -> cd {
        if (n > P || m > n || -m > n) return cd{0, 0};
        return coef[nmi(n, m)];
    };
    Dz = Dp = Dm = B = cd{0, 0};
    auto add = [&](int n, int mi, cd zv) {
        cd t = F[n + 1] * zv;
        B = cmac(B, t, coef[nmi(n, mi)]);
        if (n + 1 > P) return;
        int k1 = n + 1;
        Dz = cmac(Dz, t, __ldg(zc.g3 + nmi(k1, mi)) * c(k1, mi));
        if (mi + 1 <= k1) Dp = cmac(Dp, t, (-__ldg(zc.gp + nmi(k1, mi + 1))) * c(k1, mi + 1));
        if (mi - 1 >= -k1) Dm = cmac(Dm, t, __ldg(zc.gm + nmi(k1, mi - 1)) * c(k1, mi - 1));
    };
    for (int sgn = 0; sgn < 2; ++sgn) {
        cd xs = sgn ? xm : xp;
        cd d = {1, 0};
        for (int m = 0; m <= P; ++m) {
            if (m > 0) d = (-__ldg(zc.dg + m)) * (xs * d);
            if (sgn == 1 && m == 0) continue;
            int mi = sgn ? -m : m;
            add(m, mi, d);
            if (m + 1 > P) continue;
            cd p2 = d, p1 = __ldg(zc.s21 + m) * (z * d);
            add(m + 1, mi, p1);
            for (int n = m + 2; n <= P; ++n) {
                int k = nmi(n, m);
                cd cur = zc.A[k] * (z * p1) - zc.B[k] * (r2 * p2);
                add(n, mi, cur);
                p2 = p1;
                p1 = cur;
            }
        }
    }
}

// target gradients of M2P (List 3, S waves) and L2P (R waves), FP64, added to
// g [rhs][3][n]
__global__ void k_eval3h_grad(Exp3hArgs A, const int* __restrict__ leaves, const int* __restrict__ l3off,
                              const int* __restrict__ l3, const cd* __restrict__ mp, const cd* __restrict__ loc,
                              cd* __restrict__ g) {
    extern __shared__ cd sm[];
    int b = leaves[blockIdx.x];
    int rhs = blockIdx.y;
    int P = A.Plev[A.blevel[b]];
    int nc = (P + 1) * (P + 1);
    cd* coef = sm;
    int s0 = A.bst[b], s1 = A.ben[b];
    cd F[kH3MaxP + 3];
    for (int t0 = s0; t0 < s1; t0 += blockDim.x) {
        int i = t0 + threadIdx.x;
        bool valid = i < s1;
        cd x[3] = {{0, 0}, {0, 0}, {0, 0}};
        if (valid) load3(A.xr, A.xi, A.n, i, x);
        cd G[3] = {{0, 0}, {0, 0}, {0, 0}};
        auto accum = [&](const cd* d, int Pq) {
            cd Dz, Dp, Dm, B;
            eval_wave_grad(A.zc, d[0], d[1], d[2], Pq, F, coef, Dz, Dp, Dm, B);
            G[0] += Dp + Dm - A.kappa * (d[0] * B);
            G[1] += mul_i(Dp - Dm) - A.kappa * (d[1] * B);
            G[2] += Dz - A.kappa * (d[2] * B);
        };
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
                radial_seq(false, A.kappa, d[0] * d[0] + d[1] * d[1] + d[2] * d[2], Ps + 1, F);
                accum(d, Ps);
            }
        }
        __syncthreads();
        const cd* lc = loc + (int64_t)rhs * A.ncoef + A.eoff[b];
        for (int c = threadIdx.x; c < nc; c += blockDim.x) coef[c] = lc[c];
        __syncthreads();
        if (valid) {
            cd d[3];
            for (int a = 0; a < 3; ++a) d[a] = x[a] - cd{A.cre[3 * b + a], A.cim[3 * b + a]};
            radial_seq(true, A.kappa, d[0] * d[0] + d[1] * d[1] + d[2] * d[2], P + 1, F);
            accum(d, P);
            cd* go = g + (int64_t)rhs * 3 * A.n + i;
            for (int a = 0; a < 3; ++a) go[(int64_t)a * A.n] += G[a];
        }
    }
}

// M2P over List 3 (S waves) and L2P (R waves); one thread per target.
__global__ void k_eval3h(Exp3hArgs A, const int* __restrict__ leaves, const int* __restrict__ l3off,
                         const int* __restrict__ l3, const cd* __restrict__ mp, const cd* __restrict__ loc,
                         cd* __restrict__ u, int do_l2p) {
    extern __shared__ cd sm[];
    int b = leaves[blockIdx.x];
    int rhs = blockIdx.y;
    int P = A.Plev[A.blevel[b]];
    int nc = (P + 1) * (P + 1);
    cd* coef = sm;
    int s0 = A.bst[b], s1 = A.ben[b];
    cd F[kH3MaxP + 2];
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
                radial_seq(false, A.kappa, d[0] * d[0] + d[1] * d[1] + d[2] * d[2], Ps, F);
                acc += eval_wave(A.zc, d[0], d[1], d[2], Ps, F, coef);
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
            radial_seq(true, A.kappa, d[0] * d[0] + d[1] * d[1] + d[2] * d[2], P, F);
            acc += eval_wave(A.zc, d[0], d[1], d[2], P, F, coef);
            u[(int64_t)rhs * A.n + i] += acc;
        }
    }
}

// ---------------------------------------------------------------------------
// L2P in complex64 arithmetic (mixed precision), 3D Helmholtz and Laplace.
//
// With x~ = (x - c)/rho_b (rho_b = sqrt(3)/2 w, the leaf's radius) the local
// expansion is evaluated as
//   Helmholtz  u = sum L^_n^m jh_n(k rho) Z_n^m(x~),  L^ = L_n^m (k rho_b)^n/(2n+1)!!
//   Laplace    u = sum L^_n^m Z_n^m(x~),              L^ = L_n^m lsd_n^m rho_b^n
// (Z_n^m(x) = rho_b^n Z_n^m(x~); U_n^m = lsd_n^m Z_n^m), where
//   jh_n(z) = j_n(z) (2n+1)!!/z^n
// is entire in w = z^2 with jh_n(0) = 1, so every factor stays O(1) in FP32
// at any leaf size. From j_{n-1} + j_{n+1} = (2n+1)/z j_n,
//   jh_{n-1} = jh_n - w jh_{n+1}/((2n+1)(2n+3)),
// and the ratios q_n = jh_n/jh_{n-1} = 1/(1 - w q_{n+1}/((2n+1)(2n+3))) follow
// by Miller's backward recurrence from q = 1 far above P; jh_0 = j_0 comes
// from the plane-wave normalisation exp(-+ i z) = sum (2n+1) (-+ i)^n j_n =
// jh_0 sum (-+ i z)^n/(2n-1)!! prod_{k<=n} q_k (sign with |exp| >= 1, as in
// the FP64 Miller recurrence). The coefficients are formed in FP64 per leaf
// and rounded; each harmonic column is summed in FP32 and the columns in a
// compensated (Kahan) FP32 sum.
// ---------------------------------------------------------------------------
struct L2p3fArgs {
    const double* xr;
    const double* xi;
    int64_t n;
    const int* blevel;
    const int* bst;
    const int* ben;
    const double* cre;
    const double* cim;
    const int* Plev;
    const int64_t* eoff;
    int64_t ncoef;
    double kappa;
    double W;            // root box width
    const float* zA;     // FP32 Z recurrence coefficients by nmi(n, m >= 0)
    const float* zB;
    const float* dg;
    const float* s21;
    const int* knm;
    const double* lsd;   // Laplace: e_m / s_n^m by nmi(n, m)
};

// jh_n(z) = j_n(z) (2n+1)!!/z^n, n = 0..P, in complex64 from w = z^2 (see
// the comment above k_l2p3f): ratios by Miller's backward recurrence from 1,
// jh_0 from the plane-wave normalisation.
__device__ __forceinline__ void jhat_seq(cf w, int P, cf* G) {
    cf zz = csqrtf_p(w);
    float big = fmaxf((float)P, hypotf(zz.x, zz.y));
    int N = (int)big + 12 + (int)sqrtf(8.f * big);
    bool up = zz.y >= 0.f;                           // exp(-i z), |.| >= 1
    cf a = up ? cf{zz.y, -zz.x} : cf{-zz.y, zz.x};   // -+ i z
    cf q = {1.f, 0.f}, H = {1.f, 0.f};
    for (int nn = N; nn >= 1; --nn) {
        float den = 1.f / ((2.f * nn + 1.f) * (2.f * nn + 3.f));
        q = cinvf(cf{1.f, 0.f} - (den * w) * q);
        if (nn <= P) G[nn] = q;
        H = cf{1.f, 0.f} + (1.f / (2.f * nn - 1.f)) * (a * (q * H));
    }
    // jh_0 = exp(a) / H
    float ex = expf(a.x), sn, cs;
    sincosf(a.y, &sn, &cs);
    cf g = cf{ex * cs, ex * sn} * cinvf(H);
    G[0] = g;
    for (int nn = 1; nn <= P; ++nn) {
        g = g * G[nn];
        G[nn] = g;
    }
}

template <bool HELM>
__global__ void __launch_bounds__(128) k_l2p3f(L2p3fArgs A, const int* __restrict__ leaves,
                                                const cd* __restrict__ loc, cd* __restrict__ u) {
    extern __shared__ unsigned char smraw[];
    int b = leaves[blockIdx.x];
    int rhs = blockIdx.y;
    int lev = A.blevel[b];
    int P = A.Plev[lev];
    int nc = (P + 1) * (P + 1);
    double rb = 0.86602540378443864676 * ldexp(A.W, -lev);
    double* scl = reinterpret_cast<double*>(smraw);              // P + 1
    cf* coef = reinterpret_cast<cf*>(scl + (P + 1));             // (P + 1)^2
    if (threadIdx.x == 0) {
        double f = 1.0, g = HELM ? A.kappa * rb : rb;
        for (int n = 0; n <= P; ++n) {
            scl[n] = f;
            f *= HELM ? g / (2.0 * n + 3.0) : g;
        }
    }
    __syncthreads();
    const cd* lc = loc + (int64_t)rhs * A.ncoef + A.eoff[b];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        int n, m;
        nm_tab(A.knm, c, n, m);
        double s = scl[n];
        if (!HELM) s *= __ldg(A.lsd + c);
        coef[c] = to_cf(s * lc[c]);
    }
    __syncthreads();
    double irb = 1.0 / rb;
    cd cen[3];
    for (int a = 0; a < 3; ++a) cen[a] = cd{A.cre[3 * b + a], A.cim[3 * b + a]};
    cf G[kH3MaxP + 1];
    for (int i = A.bst[b] + threadIdx.x; i < A.ben[b]; i += blockDim.x) {
        cf x[3];
        for (int a = 0; a < 3; ++a)
            x[a] = to_cf(irb * (cd{A.xr[a * A.n + i], A.xi[a * A.n + i]} - cen[a]));
        cf xp = x[0] + mul_if(x[1]), xm = x[0] - mul_if(x[1]), z = x[2];
        cf r2 = xp * xm + z * z;
        if (HELM) {
            // w = (k rho)^2 = (k rho_b)^2 x~.x~
            float kr = (float)(A.kappa * rb);
            jhat_seq((kr * kr) * r2, P, G);
        }
        Kahan acc;
        for (int sgn = 0; sgn < 2; ++sgn) {
            cf xs = sgn ? xm : xp;
            cf d = {1.f, 0.f};
            for (int m = 0; m <= P; ++m) {
                if (m > 0) d = (-__ldg(A.dg + m)) * (xs * d);
                if (sgn == 1 && m == 0) continue;
                int mi = sgn ? -m : m;
                cf col = coef[nmi(m, mi)] * (HELM ? G[m] * d : d);
                if (m + 1 <= P) {
                    cf p2 = d, p1 = __ldg(A.s21 + m) * (z * d);
                    col = cmacf(col, coef[nmi(m + 1, mi)], HELM ? G[m + 1] * p1 : p1);
                    for (int n = m + 2; n <= P; ++n) {
                        int k = nmi(n, m);
                        cf cur = __ldg(A.zA + k) * (z * p1) - __ldg(A.zB + k) * (r2 * p2);
                        col = cmacf(col, coef[nmi(n, mi)], HELM ? G[n] * cur : cur);
                        p2 = p1;
                        p1 = cur;
                    }
                }
                acc.add(col);
            }
        }
        u[(int64_t)rhs * A.n + i] += acc.value();
    }
}

// Single-layer P2M in complex64 products (mixed precision), 3D Helmholtz and
// Laplace. With y~ = (y - c)/rho_b,
//   Helmholtz  M_n^m = i k (2n+1) (k rho_b)^n/(2n+1)!! sum s jh_n(k rho) Z_n^{-m}(y~)
//   Laplace    M_n^m = lsd_n^m rho_b^n sum s Z_n^{-m}(y~)
// (the forms of k_p2x3h_slp rewritten as in k_l2p3f). Each warp stages 32
// sources (their jh table, x+, x-, x3 and density) and then takes (source,
// harmonic column) items in rounds of 32, one per lane; a column owns the
// coefficients (n, -mu), n >= |mu|, so with 2P+1 >= 32 columns the lanes of a
// round write disjoint coefficients (fewer columns: one source at a time, a
// lane per column). Products are complex64 and each warp's accumulator row is
// a compensated (Kahan) complex64 sum; the rows are summed in warp order in
// FP64 and scaled in FP64.
constexpr int kP2m3fWarps = 4;

template <bool HELM>
__global__ void __launch_bounds__(kP2m3fWarps * 32) k_p2m3f(L2p3fArgs A, const int* __restrict__ boxes,
                                                             const cd* __restrict__ sigma, int64_t dstride,
                                                             cd* __restrict__ out) {
    extern __shared__ unsigned char smraw[];
    int b = boxes[blockIdx.x];
    int rhs = blockIdx.y;
    int lev = A.blevel[b];
    int P = A.Plev[lev];
    int nc = (P + 1) * (P + 1), C = 2 * P + 1;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4* acc = reinterpret_cast<float4*>(smraw);                         // [nwarp][nc]: sum, compensation
    cf* Gs = reinterpret_cast<cf*>(acc + (size_t)kP2m3fWarps * nc);         // [nwarp][32][P+1]
    cf* Ys = Gs + (size_t)kP2m3fWarps * 32 * (P + 1);                       // [nwarp][32][4]
    float4* accw = acc + (size_t)wid * nc;
    cf* Gw = Gs + (size_t)wid * 32 * (P + 1);
    cf* Yw = Ys + (size_t)wid * 32 * 4;
    for (int c = lane; c < nc; c += 32) accw[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    auto kadd = [&](int k, cf t) {
        float4 a = accw[k];
        float yx = t.x - a.z, tx = a.x + yx;
        float yy = t.y - a.w, ty = a.y + yy;
        accw[k] = make_float4(tx, ty, (tx - a.x) - yx, (ty - a.y) - yy);
    };
    double rb = 0.86602540378443864676 * ldexp(A.W, -lev), irb = 1.0 / rb;
    cd cen[3];
    for (int a = 0; a < 3; ++a) cen[a] = cd{A.cre[3 * b + a], A.cim[3 * b + a]};
    float kr = (float)(A.kappa * rb);
    int s0 = A.bst[b], s1 = A.ben[b];
    for (int base = s0 + wid * 32; base < s1; base += kP2m3fWarps * 32) {
        int cnt = min(32, s1 - base);
        __syncwarp();
        if (lane < cnt) {
            int j = base + lane;
            cf y[3];
            for (int a = 0; a < 3; ++a) y[a] = to_cf(irb * (cd{A.xr[a * A.n + j], A.xi[a * A.n + j]} - cen[a]));
            cf xp = y[0] + mul_if(y[1]), xm = y[0] - mul_if(y[1]);
            Yw[lane * 4 + 0] = xp;
            Yw[lane * 4 + 1] = xm;
            Yw[lane * 4 + 2] = y[2];
            Yw[lane * 4 + 3] = to_cf(sigma[rhs * dstride + j]);
            if (HELM) jhat_seq((kr * kr) * (xp * xm + y[2] * y[2]), P, Gw + lane * (P + 1));
        }
        __syncwarp();
        int items = cnt * C;
        int step = C >= 32 ? 32 : C;
        for (int r0 = 0; r0 < items; r0 += step) {
            int it = r0 + lane;
            if (lane < step && it < items) {
                int js = it / C, col = it - js * C;
                cf xp = Yw[js * 4 + 0], xm = Yw[js * 4 + 1], z = Yw[js * 4 + 2], d = Yw[js * 4 + 3];
                cf r2 = xp * xm + z * z;
                const cf* G = Gw + js * (P + 1);
                int am = col <= P ? col : col - P;
                bool neg = col > P;
                int m = neg ? am : -am;
                cf xs = neg ? xm : xp;
                for (int i = 1; i <= am; ++i) d = (-__ldg(A.dg + i)) * (xs * d);
                kadd(nmi(am, m), HELM ? G[am] * d : d);
                if (am + 1 <= P) {
                    cf p2 = d, p1 = __ldg(A.s21 + am) * (z * d);
                    kadd(nmi(am + 1, m), HELM ? G[am + 1] * p1 : p1);
                    for (int n = am + 2; n <= P; ++n) {
                        int kk = nmi(n, am);
                        cf cur = __ldg(A.zA + kk) * (z * p1) - __ldg(A.zB + kk) * (r2 * p2);
                        kadd(nmi(n, m), HELM ? G[n] * cur : cur);
                        p2 = p1;
                        p1 = cur;
                    }
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    cd* o = out + (int64_t)rhs * A.ncoef + A.eoff[b];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        cd v = {0.0, 0.0};
        for (int w = 0; w < kP2m3fWarps; ++w) {
            float4 a = acc[(size_t)w * nc + c];
            v += cd{(double)a.x - (double)a.z, (double)a.y - (double)a.w};
        }
        int n, m;
        nm_tab(A.knm, c, n, m);
        double sc = 1.0, g = HELM ? A.kappa * rb : rb;
        for (int j = 1; j <= n; ++j) sc *= HELM ? g / (2.0 * j + 1.0) : g;
        if (HELM) o[c] = mul_i((A.kappa * (2.0 * n + 1.0) * sc) * v);
        else o[c] = (__ldg(A.lsd + c) * sc) * v;
    }
}

// shared memory of k_p2m3f at order P
static size_t p2m3f_smem(int P) {
    size_t nc = (size_t)(P + 1) * (P + 1);
    return sizeof(float4) * kP2m3fWarps * nc + sizeof(cf) * (size_t)kP2m3fWarps * 32 * (P + 1 + 4);
}

static void launch_p2m3f(H3Tables* TB, bool helm, cfmm_plan_s* P, const int* boxes, int cnt, int PL,
                         const int* dPlev, const int64_t* eoff, int64_t ncoef, const cd* sigma, int64_t dstride,
                         cd* out, int nrhs) {
    if (cnt <= 0) return;
    TreeDev& T = P->tree;
    L2p3fArgs A{P->xr.get(), P->xi.get(), P->n, T.level.get(), T.start.get(), T.end.get(), T.cen_re.get(),
                T.cen_im.get(), dPlev, eoff, ncoef, P->kappa, P->W, TB->zAf.get(), TB->zBf.get(),
                TB->dgf.get(), TB->s21f.get(), TB->knm.get(), TB->lsd.get()};
    size_t smem = p2m3f_smem(PL);
    dim3 g((unsigned)cnt, nrhs);
    if (helm) {
        if (smem > 48 * 1024) CFMM_CUDA(cudaFuncSetAttribute(k_p2m3f<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_p2m3f<true><<<g, kP2m3fWarps * 32, smem, P->stream>>>(A, boxes, sigma, dstride, out);
    } else {
        if (smem > 48 * 1024) CFMM_CUDA(cudaFuncSetAttribute(k_p2m3f<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_p2m3f<false><<<g, kP2m3fWarps * 32, smem, P->stream>>>(A, boxes, sigma, dstride, out);
    }
    CFMM_LAUNCHED();
}

static void launch_l2p3f(H3Tables* TB, bool helm, cfmm_plan_s* P, const int* leaves, int cnt, int maxP,
                         const int* dPlev, const int64_t* eoff, int64_t ncoef, const cd* loc, cd* u, int nrhs) {
    if (cnt == 0) return;
    TreeDev& T = P->tree;
    L2p3fArgs A{P->xr.get(), P->xi.get(), P->n, T.level.get(), T.start.get(), T.end.get(), T.cen_re.get(),
                T.cen_im.get(), dPlev, eoff, ncoef, P->kappa, P->W, TB->zAf.get(), TB->zBf.get(),
                TB->dgf.get(), TB->s21f.get(), TB->knm.get(), TB->lsd.get()};
    size_t smem = sizeof(double) * (size_t)(maxP + 1) + sizeof(cf) * (size_t)(maxP + 1) * (maxP + 1);
    dim3 g((unsigned)cnt, nrhs);
    if (helm) k_l2p3f<true><<<g, 128, smem, P->stream>>>(A, leaves, loc, u);
    else k_l2p3f<false><<<g, 128, smem, P->stream>>>(A, leaves, loc, u);
    CFMM_LAUNCHED();
}

// ---------------------------------------------------------------------------
// translations
// ---------------------------------------------------------------------------
struct Tr3hArgs {
    const double* cre;
    const double* cim;
    const int64_t* eoff;
    int64_t ncoef;
    const double* Dh;
    const int64_t* Dhoff;
    const double* inv2n1;
    const double* al;
    const double* be;
    const double* ibe;
    const double* mu;
    const double* nu;
    const int* knm;
    double kappa;
    // source enumeration (mode 0: children cbeg..cend; 1: List 2; 2: parent)
    const int* cbeg;
    const int* cend;
    const int* loff;
    const int* lent;
    const int* parent;
    const int* leaf;
    const int* qbox;     // owner (destination) box of each List-2 entry
};

// i^e x for integer e (a permutation of the parts; no arithmetic)
__device__ __forceinline__ cd mul_ipow(int e, cd x) {
    switch (e & 3) {
        case 0: return x;
        case 1: return cd{-x.y, x.x};
        case 2: return cd{-x.x, -x.y};
        default: return cd{x.y, -x.x};
    }
}

// The fixed matrices D_n satisfy D[-m][m'] = D[m][-m'] = (-1)^{n+m+m'} D[m][m']
// and D^T = S D S, S = diag((-1)^m). With w+-_{m'} = x_{m'} +- (-1)^{m'} x_{-m'}
// (m' > 0), row m >= 0 of D x and row -m follow from one half-row pass:
//   n+m even:  y_{+-m} = D[m][0] x_0 + E +- O,   E, O = sum over even / odd m' > 0 of D[m][m'] w+_{m'}
//   n+m odd:   y_m = E + O,  y_{-m} = O - E      (with w-; D[m][0] = 0)
// Dh holds D[m][m'] for m, m' >= 0, column-major per order (Dh_n[m' (n+1) + m]).

// w-pass: wb <- w+- of x, x_k = f_k in_k with the per-coefficient factor f
// given by (i-power, sign, power table): x = i^{ip*m} sg^m pw[m + Pm] in
__device__ __forceinline__ void w_pass(const int* knm, const cd* in, cd* wb, int P, int ip, int sgn_alt,
                                       const cd* pw, int Pm) {
    int W = (P + 1) * (P + 2) / 2;          // items (n, m >= 0)
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        int n = (int)((sqrtf(8.0f * w + 1.0f) - 1.0f) * 0.5f);
        while ((n + 1) * (n + 2) / 2 <= w) ++n;
        while (n * (n + 1) / 2 > w) --n;
        int m = w - n * (n + 1) / 2;
        int k = nmi(n, m);
        auto xf = [&](int mm) {
            cd v = in[nmi(n, mm)];
            if (pw) v = v * pw[mm + Pm];
            v = mul_ipow(ip * mm, v);
            if (sgn_alt && (mm & 1)) v = -v;
            return v;
        };
        cd xp = xf(m);
        if (m == 0) {
            wb[k] = xp;
            continue;
        }
        cd xm = xf(-m);
        if (m & 1) xm = -xm;
        wb[nmi(n, m)] = xp + xm;
        wb[nmi(n, -m)] = xp - xm;
    }
}

// D-pass: y = D x from the w+- of x; out_k = g_k y_k with g = i^{op*m} (sgn_out:
// times (-1)^m), optionally times pw_out[m + Pm], accumulated when acc != 0
__device__ __forceinline__ void d_pass(const double* Dh, const int64_t* Dhoff, const cd* wb, cd* out, int P,
                                       int op, int sgn_out, const cd* pwo, int Pm, int accum) {
    int W = (P + 1) * (P + 2) / 2;          // work items (n, m >= 0)
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        int n = (int)((sqrtf(8.0f * w + 1.0f) - 1.0f) * 0.5f);
        while ((n + 1) * (n + 2) / 2 <= w) ++n;
        while (n * (n + 1) / 2 > w) --n;
        int m = w - n * (n + 1) / 2;
        const double* Dn = Dh + __ldg(Dhoff + n);
        int N1 = n + 1;
        bool odd = (n + m) & 1;
        cd E = {0, 0}, O = {0, 0};
        const cd* wv = wb + n * n + n;       // wv[m'] = w+_{m'}, wv[-m'] = w-_{m'}
        for (int mp = 1; mp <= n; ++mp) {
            double d = Dn[mp * N1 + m];
            cd wq = odd ? wv[-mp] : wv[mp];
            if (mp & 1) O = rmac(O, d, wq);
            else E = rmac(E, d, wq);
        }
        cd yp, ym;
        if (odd) {
            yp = E + O;
            ym = O - E;
        } else {
            cd d0 = Dn[m] * wv[0];
            yp = d0 + E + O;
            ym = d0 + E - O;
        }
        auto emit = [&](int mm, cd y) {
            y = mul_ipow(op * mm, y);
            if (sgn_out && (mm & 1)) y = -y;
            if (accum && pwo) {
                out[nmi(n, mm)] = cmac(out[nmi(n, mm)], y, pwo[mm + Pm]);
                return;
            }
            if (pwo) y = y * pwo[mm + Pm];
            if (accum) out[nmi(n, mm)] += y;
            else out[nmi(n, mm)] = y;
        };
        emit(m, yp);
        if (m > 0) emit(-m, ym);
    }
}

// The fixed real rotation Q_k (k = 0, 1) of the fixed-frame translation,
// applied in place to the coefficients x (order P) through wb and tmp: the
// rotation sequence of the translation kernels with e = i^k and alpha = pi/2,
// whose diagonal factors are powers of i (no tables). Ends with a barrier.
__device__ void rot_fixed(const Tr3hArgs& A, const double* Dh, cd* x, cd* wb, cd* tmp, int P, int Pm, int k) {
    w_pass(A.knm, x, wb, P, 1 + k, 0, nullptr, Pm);
    __syncthreads();
    d_pass(Dh, A.Dhoff, wb, tmp, P, 0, 0, nullptr, Pm, 0);
    __syncthreads();
    w_pass(A.knm, tmp, wb, P, 3, 0, nullptr, Pm);
    __syncthreads();
    d_pass(Dh, A.Dhoff, wb, x, P, 1, 0, nullptr, Pm, 0);
    __syncthreads();
}

// Its inverse from x into out (added when accum != 0); x and tmp are
// overwritten. Needs a barrier before (x written) and leaves out unsynchronised.
__device__ void rot_fixed_inv(const Tr3hArgs& A, const double* Dh, cd* x, cd* wb, cd* tmp, cd* out, int P, int Pm,
                              int k, int accum) {
    w_pass(A.knm, x, wb, P, 1, 0, nullptr, Pm);
    __syncthreads();
    d_pass(Dh, A.Dhoff, wb, tmp, P, 0, 0, nullptr, Pm, 0);
    __syncthreads();
    w_pass(A.knm, tmp, wb, P, 1, 0, nullptr, Pm);
    __syncthreads();
    d_pass(Dh, A.Dhoff, wb, out, P, (1 - k) & 3, 0, nullptr, Pm, accum);
}

// Per-shift quantities of a launch, one thread per (destination, source)
// pair: e = e^{i beta}, e_a = e^{i alpha} and f_l(kappa t), l <= NR. Pair p
// of the launch is list entry qfirst + p (mode 1), child box qfirst + p
// (mode 0) or destination box lo + p (mode 2).
__global__ void k_tr3h_pre(Tr3hArgs A, int mode, int lo, int qfirst, int npair, int NR, int use_h,
                           cd* __restrict__ sc, cd* __restrict__ fl, int* __restrict__ fb, int Pm,
                           cd* __restrict__ pwt) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npair) return;
    int b, s;
    if (mode == 1) {
        int q = qfirst + p;
        s = A.lent[q];
        b = A.qbox[q];
    } else if (mode == 0) {
        s = qfirst + p;
        b = A.parent[s];
    } else {
        b = lo + p;
        s = A.parent[b];
    }
    cd d[3];
    for (int k = 0; k < 3; ++k) d[k] = cd{A.cre[3 * b + k] - A.cre[3 * s + k], A.cim[3 * b + k] - A.cim[3 * s + k]};
    cd s2 = d[0] * d[0] + d[1] * d[1];
    // an isotropic complex direction in the xy-plane (s^2 = 0 or nearly, with
    // (d1, d2) != 0) has no z-rotation angle: the pair is translated in the
    // frame of the fixed real rotation Q_k (Q_0 d = (-d3, d2, d1), Q_1 d =
    // (-d3, -d1, d2)), the one with the larger |(Q d)_1^2 + (Q d)_2^2|
    int fr = -1;
    {
        double n2 = cabs2(d[0]) + cabs2(d[1]) + cabs2(d[2]);
        bool xy = d[0].x != 0.0 || d[0].y != 0.0 || d[1].x != 0.0 || d[1].y != 0.0;
        if (xy && cabs2(s2) <= (kDegenTol * n2) * (kDegenTol * n2)) {
            cd a0 = d[2] * d[2] + d[1] * d[1], a1 = d[2] * d[2] + d[0] * d[0];
            fr = cabs2(a0) >= cabs2(a1) ? 0 : 1;
            cd q1 = fr == 0 ? d[1] : -d[0], q2 = fr == 0 ? d[0] : d[1];
            d[0] = -d[2];
            d[1] = q1;
            d[2] = q2;
            s2 = d[0] * d[0] + d[1] * d[1];
        }
    }
    fb[p] = fr;
    cd t = csqrt_p(s2 + d[2] * d[2]);
    cd sq = {0, 0}, e = {1, 0};
    if (!(s2.x == 0.0 && s2.y == 0.0)) {
        sq = csqrt_p(s2);
        e = (d[0] + mul_i(d[1])) / sq;
    }
    cd ea = (d[2] + mul_i(sq)) / t;
    sc[2 * (size_t)p] = e;
    sc[2 * (size_t)p + 1] = ea;
    if (pwt) {
        // e^m and e_a^m for m in [-Pm, Pm] (running products), for the
        // translation kernel's diagonal factors
        int W = 2 * Pm + 1;
        cd* pe = pwt + (size_t)p * 2 * W;
        for (int q = 0; q < 2; ++q) {
            cd* dst = pe + q * W;
            cd x = q ? ea : e, ix = cinv(x), v = {1, 0}, iv = {1, 0};
            dst[Pm] = v;
            for (int m = 1; m <= Pm; ++m) {
                v = v * x;
                iv = iv * ix;
                dst[Pm + m] = v;
                dst[Pm - m] = iv;
            }
        }
    }
    if (NR < 0) {                      // Laplace: only t
        fl[p] = t;
        return;
    }
    cd* f = fl + (size_t)p * (NR + 1);
    cd z = A.kappa * t;
    if (use_h) sph_h_seq(z, NR, f);
    else sph_j_seq(z, NR, f);
}

// x^m for m = 0..M by binary exponentiation (one lane per m)
__device__ __forceinline__ cd cpow_int(cd x, int m) {
    cd r = {1, 0};
    while (m) {
        if (m & 1) r = r * x;
        x = x * x;
        m >>= 1;
    }
    return r;
}

// Coaxial translation with the work flattened over the block (equal input
// and output orders P, all columns of T^m in shared memory at once):
//   1. the columns of every m advance together: at step c' thread items are
//      the (m, row) pairs of column c = m + c' + 1 (rows c..NR-c, NR = 2P),
//      from the two previous columns of the same m (the recurrence of the
//      file comment, in the stable direction);
//   2. rows <= P of each column go to a compact lower triangle per m
//      (rows r = m..P, columns c = m..r, at (r-m)(r-m+1)/2 + c - m, m-blocks
//      one after the other);
//   3. the product out_n^{+-m} = sum_{c<=n} T_{n c} a_c + (2n+1)(-1)^n
//      sum_{r>n} T_{r n} a~_r, one thread item per (m, n, sign), m-major, so
//      the lanes of a warp share a loop length.
// The per-warp path below does the same work with one warp per m, whose lanes
// idle as the columns shorten.
__host__ __device__ inline size_t tr3h_tri_off(int P, int m) {
    size_t o = 0;
    for (int q = 0; q < m; ++q) o += (size_t)(P - q + 1) * (P - q + 2) / 2;
    return o;
}
// g_c = (-1)^c (2c + 1), the column factor of the stored coaxial triangles
__device__ __forceinline__ double coax_g(int c) { return (c & 1) ? -(2.0 * c + 1.0) : (2.0 * c + 1.0); }
__host__ __device__ inline size_t tr3h_tri_size(int P) { return (size_t)(P + 1) * (P + 2) * (P + 3) / 6; }
__host__ __device__ inline size_t tr3h_flat_cols(int P) {
    return (size_t)3 * (P + 1) * (2 * P + 2) + tr3h_tri_off(P, P + 1);
}

// out_n^{+-m} = sum_{c<=n} T_{n c} a_c + (2n+1)(-1)^n sum_{r>n} T_{r n} a~_r from
// the compact triangles tri (shared or global memory) holding T'_{r c} =
// g_c T_{r c}, g_c = (-1)^c (2c+1): with a~_c = a_c / g_c both sums read the same
// vector a~, out_n = sum_{c<=n} T'_{n c} a~_c + sum_{r>n} T'_{r n} a~_r, one loop of
// P - m + 1 terms for every n of a given m (row n of the triangle, then its
// column n). One thread item per (m >= 0, n) computes both signs of m from the
// same operator entries and writes them as the first pass of the back rotation
// would (w+- of Phi out, see w_pass), so that pass is not run. m-major items.
__device__ void coax_product_w(int P, const cd* __restrict__ tri, const cd* __restrict__ wb, cd* __restrict__ wout) {
    int nitem = (P + 1) * (P + 2) / 2;
    for (int t = threadIdx.x; t < nitem; t += blockDim.x) {
        int m = 0, rem = t;
        while (rem >= P - m + 1) {
            rem -= P - m + 1;
            ++m;
        }
        int n = m + rem;
        const cd* T = tri + tr3h_tri_off(P, m);
        const int k0 = n - m;                               // row n holds columns m..n
        const int rowb = k0 * (k0 + 1) / 2;
        cd sp = {0, 0}, sn = {0, 0};
        for (int j = 0; j <= P - m; ++j) {
            int idx, k;
            if (j <= k0) {
                idx = rowb + j;                             // T'_{n, m+j}
                k = m + j;
            } else {
                int r = n + (j - k0);                       // T'_{r, n}
                idx = (r - m) * (r - m + 1) / 2 + k0;
                k = r;
            }
            cd tv = T[idx];
            sp = cmac(sp, tv, wb[nmi(k, m)]);
            if (m > 0) sn = cmac(sn, tv, wb[nmi(k, -m)]);
        }
        // w+- of x = Phi out: x_{+-m} = i^{+-m} out_{+-m}
        cd xp = mul_ipow(m, sp);
        if (m == 0) {
            wout[nmi(n, 0)] = xp;
            continue;
        }
        cd xm = mul_ipow(-m, sn);
        if (m & 1) xm = -xm;
        wout[nmi(n, m)] = xp + xm;
        wout[nmi(n, -m)] = xp - xm;
    }
}

__device__ void coax_flat(const Tr3hArgs& A, int P, int NR, const cd* __restrict__ sect, cd* __restrict__ cols,
                          const cd* __restrict__ a, const cd* __restrict__ wb, cd* __restrict__ bb) {
    const int L = NR + 2;                       // column length
    cd* tri = cols + (size_t)3 * (P + 1) * L;
    auto col = [&](int k, int m) { return cols + ((size_t)k * (P + 1) + m) * L; };
    // columns c = m (sectorial) in buffer 1, c = m - 1 (zero) in buffer 0
    for (int t = threadIdx.x; t < (P + 1) * L; t += blockDim.x) {
        int m = t / L, r = t - m * L;
        col(0, m)[r] = cd{0, 0};
        col(1, m)[r] = (r >= m && r <= NR - m) ? sect[(size_t)m * (NR + 1) + r] : cd{0, 0};
    }
    __syncthreads();
    // column c = m into the triangles (rows m..P)
    for (int t = threadIdx.x; t < (P + 1) * (P + 1); t += blockDim.x) {
        int m = t / (P + 1), r = t - m * (P + 1);
        if (r >= m) tri[tr3h_tri_off(P, m) + (size_t)(r - m) * (r - m + 1) / 2] = coax_g(m) * col(1, m)[r];
    }
    int kp = 0, kc = 1, kn = 2;
    for (int cp = 0; cp < P; ++cp) {
        // items (m, r): m <= P - 1 - cp, r in [m + cp + 1, NR - m - cp - 1]
        int K = NR - 2 * cp - 1;                // rows of m = 0
        int nitem = 0;
        for (int m = 0; m <= P - 1 - cp; ++m) nitem += K - 2 * m;
        for (int t = threadIdx.x; t < nitem; t += blockDim.x) {
            int m = 0, rem = t;
            while (rem >= K - 2 * m) {
                rem -= K - 2 * m;
                ++m;
            }
            int c = m + cp, r = c + 1 + rem;
            const cd* prv = col(kp, m);
            const cd* cur = col(kc, m);
            double ac = __ldg(A.al + nmi(c, m)), ib = __ldg(A.ibe + nmi(c, m));
            cd v = rmac(ac * prv[r], -__ldg(A.al + nmi(r + 1, m)), cur[r + 1]);
            v = rmac(v, __ldg(A.be + nmi(r - 1, m)), cur[r - 1]);
            col(kn, m)[r] = ib * v;
        }
        __syncthreads();
        // rows c + 1 .. P of column c + 1 into the triangles
        int ns = 0;
        for (int m = 0; m <= P - 1 - cp; ++m) ns += P - (m + cp);
        for (int t = threadIdx.x; t < ns; t += blockDim.x) {
            int m = 0, rem = t;
            while (rem >= P - (m + cp)) {
                rem -= P - (m + cp);
                ++m;
            }
            int c1 = m + cp + 1, r = c1 + rem;
            tri[tr3h_tri_off(P, m) + (size_t)(r - m) * (r - m + 1) / 2 + (c1 - m)] = coax_g(c1) * col(kn, m)[r];
        }
        int k0 = kp;
        kp = kc;
        kc = kn;
        kn = k0;
    }
    __syncthreads();
    coax_product_w(P, tri, wb, bb);
}

// The coaxial operators of the M2L pairs of a launch (equal orders P), built
// once per pair for every right-hand side: one block per pair writes the
// compact triangles T^m (the layout of tr3h_tri_off, tr3h_tri_size entries)
// to tri. The sectorial columns T_{r m}^m (r = m..NR - m) come from the
// recurrence over m (one step per m, rows over the block's threads), then the
// columns of every m advance together, two buffers per m: the next column
// overwrites the one before the current one in place (each row reads only its
// own entry of it). Shared memory: the radial sequence, 2 (P+1) (NR+2)
// complex values and P+1 offsets.
__global__ void k_tr3h_tri(Tr3hArgs A, int P, int npair, const cd* __restrict__ fl, cd* __restrict__ tri) {
    extern __shared__ cd sm[];
    const int NR = 2 * P, L = NR + 2;
    cd* f = sm;
    cd* cols = f + (NR + 1);
    int* moff = (int*)(cols + (size_t)2 * (P + 1) * L);
    auto col = [&](int k, int m) { return cols + ((size_t)k * (P + 1) + m) * L; };
    const size_t tsz = tr3h_tri_size(P);
    for (int p = blockIdx.x; p < npair; p += gridDim.x) {
        __syncthreads();
        cd* T = tri + (size_t)p * tsz;
        for (int l = threadIdx.x; l <= NR; l += blockDim.x) f[l] = fl[(size_t)p * (NR + 1) + l];
        for (int m = threadIdx.x; m <= P; m += blockDim.x) moff[m] = (int)tr3h_tri_off(P, m);
        for (int t = threadIdx.x; t < 2 * (P + 1) * L; t += blockDim.x) cols[t] = cd{0, 0};
        __syncthreads();
        // sectorial columns into buffer 1 (buffer 0 stays zero: the column
        // before the first)
        for (int r = threadIdx.x; r <= NR; r += blockDim.x) {
            double sg = (r & 1) ? -1.0 : 1.0;
            col(1, 0)[r] = (sg * (2.0 * r + 1.0)) * f[r];
        }
        __syncthreads();
        for (int m = 1; m <= P; ++m) {
            const cd* pv = col(1, m - 1);
            cd* cur = col(1, m);
            int mm = m - 1;
            double inu = 1.0 / __ldg(A.nu + nmi(mm, mm));
            for (int r = m + threadIdx.x; r <= NR - m; r += blockDim.x) {
                double mu1 = __ldg(A.mu + nmi(r + 1, mm)), nu1 = __ldg(A.nu + nmi(r - 1, mm));
                cur[r] = inu * (mu1 * pv[r + 1] + nu1 * pv[r - 1]);
            }
            __syncthreads();
        }
        // column c = m of every m into the triangles (rows m..P)
        for (int t = threadIdx.x; t < (P + 1) * (P + 1); t += blockDim.x) {
            int m = t / (P + 1), r = t - m * (P + 1);
            if (r >= m) T[moff[m] + (r - m) * (r - m + 1) / 2] = coax_g(m) * col(1, m)[r];
        }
        int kp = 0, kc = 1;
        for (int cp = 0; cp < P; ++cp) {
            // items (m, r): m <= P - 1 - cp, r in [m + cp + 1, NR - m - cp - 1]
            int K = NR - 2 * cp - 1;
            int nitem = (P - cp) * (K - (P - 1 - cp));
            for (int t = threadIdx.x; t < nitem; t += blockDim.x) {
                int m = 0, rem = t;
                while (rem >= K - 2 * m) {
                    rem -= K - 2 * m;
                    ++m;
                }
                int c = m + cp, r = c + 1 + rem;
                cd* prv = col(kp, m);
                const cd* cur = col(kc, m);
                double ac = __ldg(A.al + nmi(c, m)), ib = __ldg(A.ibe + nmi(c, m));
                cd v = rmac(ac * prv[r], -__ldg(A.al + nmi(r + 1, m)), cur[r + 1]);
                v = rmac(v, __ldg(A.be + nmi(r - 1, m)), cur[r - 1]);
                prv[r] = ib * v;
            }
            __syncthreads();
            // rows c + 1 .. P of column c + 1 into the triangles
            int ns = 0;
            for (int m = 0; m <= P - 1 - cp; ++m) ns += P - (m + cp);
            for (int t = threadIdx.x; t < ns; t += blockDim.x) {
                int m = 0, rem = t;
                while (rem >= P - (m + cp)) {
                    rem -= P - (m + cp);
                    ++m;
                }
                int c1 = m + cp + 1, r = c1 + rem;
                T[moff[m] + (r - m) * (r - m + 1) / 2 + (c1 - m)] = coax_g(c1) * col(kp, m)[r];
            }
            int k0 = kp;
            kp = kc;
            kc = k0;
        }
    }
}

// One translation per destination box and source; the destination box's
// result is accumulated in shared memory and written (mode 0, 1) or added
// (mode 2) at the end. Shared layout: acc[Ko], a[Km], bb[Km], wb[Km],
// f[Pi+Po+1], pw_e[2Pm+1], pw_a[2Pm+1], pw_ai[2Pm+1], pw_ei[2Pm+1],
// sect[(Pmin+1)(Pi+Po+1)], per-warp columns [nwarps][3][Pi+Po+2] (these two
// in global scratch for large orders), then (when it fits) the Dh table.
__global__ void k_tr3h(Tr3hArgs A, int mode, int lo, int nb, int Pi, int Po, int use_h, int d_in_smem,
                       cd* __restrict__ gscr, const cd* __restrict__ in, cd* __restrict__ out, int chunk,
                       cd* __restrict__ part, int qfirst, const cd* __restrict__ pwt, const cd* __restrict__ fl,
                       int nrhs, int nchunk, int acc_glob, int flat, const int* __restrict__ fb,
                       int ops_g, const cd* __restrict__ trig) {
    extern __shared__ cd sm[];
    int Pm = max(Pi, Po), Pn = min(Pi, Po);
    int Ki = (Pi + 1) * (Pi + 1), Ko = (Po + 1) * (Po + 1), Km = (Pm + 1) * (Pm + 1);
    int NR = Pi + Po;                   // rows 0..NR
    int nwarp = blockDim.x >> 5, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // acc_glob (the largest orders): the destination accumulator lives after the
    // work arrays in the block's global scratch slice
    cd* acc = sm;
    cd* a = acc_glob ? sm : acc + Ko;
    cd* bb = a + Km;
    cd* wb = bb + Km;
    cd* f = wb + Km;
    cd* pwe = f + (NR + 1);
    cd* pwa = pwe + (2 * Pm + 1);
    cd* pwai = pwa + (2 * Pm + 1);
    cd* pwei = pwai + (2 * Pm + 1);
    cd* sect = pwei + (2 * Pm + 1);
    cd* cols = sect + (size_t)(Pn + 1) * (NR + 1);
    size_t wsz = flat ? tr3h_flat_cols(Po) : (size_t)nwarp * ((size_t)3 * (NR + 2) + (size_t)(Pm + 1) * (Pn + 1));
    double* Dsm = (double*)(cols + wsz);
    // ops_g: the coaxial operators come from trig (the launch was sized without
    // coaxial work arrays, also when it has no pairs and trig is null)
    if (ops_g) Dsm = (double*)(pwei + (2 * Pm + 1));
    if (gscr) {
        // large orders: the coaxial work arrays live in this block's slice of
        // global scratch instead of shared memory
        size_t per = (size_t)(Pn + 1) * (NR + 1) + wsz + (acc_glob ? (size_t)Ko : 0);
        sect = gscr + (size_t)blockIdx.x * per;
        cols = sect + (size_t)(Pn + 1) * (NR + 1);
        if (acc_glob) acc = cols + wsz;
        Dsm = (double*)(pwei + (2 * Pm + 1));
    }
    const double* Dh = A.Dh;
    if (d_in_smem) {
        int64_t nd = __ldg(A.Dhoff + Pm + 1);
        for (int64_t k = threadIdx.x; k < nd; k += blockDim.x) Dsm[k] = A.Dh[k];
        Dh = Dsm;
    }
    // work items (destination box, rhs, list chunk), grid-stride: a block's
    // global scratch slice is reused by its items
    int64_t nitem = (int64_t)nb * nrhs * nchunk;
    for (int64_t item = blockIdx.x; item < nitem; item += gridDim.x) {
    // with operators from trig the right-hand sides of a box are neighbours,
    // so the blocks that read a pair's operators run close together (L2)
    int bx = ops_g ? (int)((item / nrhs) % nb) : (int)(item % nb);
    int rhs = ops_g ? (int)(item % nrhs) : (int)((item / nb) % nrhs);
    int zc = (int)(item / ((int64_t)nb * nrhs));
    int b = lo + bx;
    if (mode == 0 && A.leaf[b]) continue;    // a leaf keeps its P2M expansion
    __syncthreads();
    for (int k = threadIdx.x; k < Ko; k += blockDim.x) acc[k] = cd{0, 0};
    int qa, qb;
    if (mode == 0) {
        qa = A.cbeg[b];
        qb = A.cend[b];
    } else if (mode == 1) {
        qa = A.loff[b];
        qb = A.loff[b + 1];
        if (part) {
            // chunked List 2: this block takes entries [qa + z chunk, qa + (z+1) chunk)
            qa += zc * chunk;
            qb = min(qb, qa + chunk);
        }
    } else {
        qa = 0;
        qb = 1;
    }
    for (int q = qa; q < qb; ++q) {
        int s = mode == 0 ? q : mode == 1 ? A.lent[q] : A.parent[b];
        __syncthreads();
        // shift d = c_new - c_old: M2M new = parent b, old = child s; M2L new =
        // target b, old = source s; L2L new = child b, old = parent s
        // this pair's index in the launch's prologue arrays
        int p = mode == 1 ? q - qfirst : mode == 0 ? q - qfirst : b - lo;
        const cd* src = in + (int64_t)rhs * A.ncoef + A.eoff[s];
        for (int k = threadIdx.x; k < Ki; k += blockDim.x) a[k] = src[k];
        if (!ops_g)
            for (int l = threadIdx.x; l <= NR; l += blockDim.x) f[l] = fl[(size_t)p * (NR + 1) + l];
        {
            // powers of e and e_a, m in [-Pm, Pm], from the prologue (pwe and pwa
            // are adjacent)
            const cd* pt = pwt + (size_t)p * 2 * (2 * Pm + 1);
            for (int k = threadIdx.x; k < 2 * (2 * Pm + 1); k += blockDim.x) pwe[k] = pt[k];
        }
        __syncthreads();
        for (int m = threadIdx.x - Pm; m <= Pm; m += blockDim.x) {
            pwai[Pm + m] = pwa[Pm - m];
            pwei[Pm + m] = pwe[Pm - m];
        }
        // (0) a pair in the fixed frame: turn the input into it
        int fr = __ldg(fb + p);
        if (fr >= 0) rot_fixed(A, Dh, a, wb, bb, Pi, Pm, fr);
        // (1) forward rotation: x = Phi E(e) c; y = D x; x' = S E(e_a) y; u = D x'; c~ = i^m u
        w_pass(A.knm, a, wb, Pi, 1, 0, pwe, Pm);
        __syncthreads();
        d_pass(Dh, A.Dhoff, wb, bb, Pi, 0, 0, nullptr, Pm, 0);
        __syncthreads();
        w_pass(A.knm, bb, wb, Pi, 0, 1, pwa, Pm);
        __syncthreads();
        d_pass(Dh, A.Dhoff, wb, a, Pi, 1, 0, nullptr, Pm, 0);
        // (2) coaxial: a~ = (-1)^r a / (2r+1) for the symmetric half; sectorial
        // columns (warp 0), then one warp per m
        __syncthreads();
        for (int k = threadIdx.x; k < Ki; k += blockDim.x) {
            int n, m;
            nm_tab(A.knm, k, n, m);
            double sc = __ldg(A.inv2n1 + n);
            wb[k] = ((n & 1) ? -sc : sc) * a[k];
        }
        for (int k = threadIdx.x; k < Ko; k += blockDim.x) bb[k] = cd{0, 0};
        if (wid == 0 && !ops_g) {
            for (int r = lane; r <= NR; r += 32) {
                double sg = (r & 1) ? -1.0 : 1.0;
                sect[r] = (sg * (2.0 * r + 1.0)) * f[r];
            }
            __syncwarp();
            for (int m = 1; m <= Pn; ++m) {
                const cd* pv = sect + (size_t)(m - 1) * (NR + 1);
                cd* cur = sect + (size_t)m * (NR + 1);
                int mm = m - 1;
                double inu = 1.0 / __ldg(A.nu + nmi(mm, mm));
                for (int r = m + lane; r <= NR - m; r += 32) {
                    double mu1 = __ldg(A.mu + nmi(r + 1, mm)), nu1 = __ldg(A.nu + nmi(r - 1, mm));
                    cur[r] = inu * (mu1 * pv[r + 1] + nu1 * pv[r - 1]);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (ops_g) {
            coax_product_w(Po, trig + (size_t)p * tr3h_tri_size(Po), wb, bb);
        } else if (flat) {
            coax_flat(A, Po, NR, sect, cols, a, wb, bb);
        } else
        for (int m = wid; m <= Pn; m += nwarp) {
            cd* cm1 = cols + (size_t)wid * ((size_t)3 * (NR + 2) + (size_t)(Pm + 1) * (Pn + 1));
            cd* c0 = cm1 + (NR + 2);
            cd* c1 = c0 + (NR + 2);
            cd* Tm = c1 + (NR + 2);              // lower triangle T[r][c], r <= Pm, c <= Pn
            const cd* sc = sect + (size_t)m * (NR + 1);
            for (int r = lane; r <= NR; r += 32) {
                cm1[r] = cd{0, 0};
                c0[r] = (r >= m && r <= NR - m) ? sc[r] : cd{0, 0};
            }
            __syncwarp();
            for (int c = m; c <= Pn; ++c) {
                // column c holds T_{r,c} for rows c <= r <= NR - c; keep rows <= Pm
                for (int r = c + lane; r <= Pm; r += 32) Tm[r * (Pn + 1) + c] = c0[r];
                if (c == Pn) break;
                // next column c + 1, rows c + 1 .. NR - c - 1
                double ac = __ldg(A.al + nmi(c, m)), ib = __ldg(A.ibe + nmi(c, m));
                for (int r = c + 1 + lane; r <= NR - c - 1; r += 32) {
                    cd v = rmac(ac * cm1[r], -__ldg(A.al + nmi(r + 1, m)), c0[r + 1]);
                    if (r - 1 >= m) v = rmac(v, __ldg(A.be + nmi(r - 1, m)), c0[r - 1]);
                    c1[r] = ib * v;
                }
                __syncwarp();
                cd* tmp = cm1;
                cm1 = c0;
                c0 = c1;
                c1 = tmp;
            }
            __syncwarp();
            // out_n^{mm} = sum_{c <= min(n, Pi)} T_{n c} a_c^{mm}
            //            + (2n+1)(-1)^n sum_{n < r <= Pi} T_{r n} a~_r^{mm},  mm = +-m;
            // one lane per (n, sign)
            int nout = Po - m + 1, nitems = m > 0 ? 2 * nout : nout;
            for (int it = lane; it < nitems; it += 32) {
                int n = m + (it % nout);
                int mm = it < nout ? m : -m;
                cd sp = {0, 0};
                int ce = min(n, Pi);
                const cd* Tr = Tm + n * (Pn + 1);
                for (int c = m; c <= ce; ++c) sp = cmac(sp, Tr[c], a[nmi(c, mm)]);
                if (n < Pi) {
                    cd up = {0, 0};
                    for (int r = n + 1; r <= Pi; ++r) up = cmac(up, Tm[r * (Pn + 1) + n], wb[nmi(r, mm)]);
                    double g = (n & 1) ? -(2.0 * n + 1.0) : (2.0 * n + 1.0);
                    sp += g * up;
                }
                bb[nmi(n, mm)] = sp;
            }
        }
        __syncthreads();
        // (3) back rotation: x = Phi c'; y = D x; x' = S E(1/e_a) y; u = D x'; acc += E(1/e) i^m u
        // (the flat and operator paths left w+- of Phi c' in bb already)
        if (ops_g || flat) {
            d_pass(Dh, A.Dhoff, bb, a, Po, 0, 0, nullptr, Pm, 0);
        } else {
            w_pass(A.knm, bb, wb, Po, 1, 0, nullptr, Pm);
            __syncthreads();
            d_pass(Dh, A.Dhoff, wb, a, Po, 0, 0, nullptr, Pm, 0);
        }
        __syncthreads();
        w_pass(A.knm, a, wb, Po, 0, 1, pwai, Pm);
        __syncthreads();
        if (fr >= 0) {
            // (4) out of the fixed frame, added to the accumulator
            d_pass(Dh, A.Dhoff, wb, a, Po, 1, 0, pwei, Pm, 0);
            __syncthreads();
            rot_fixed_inv(A, Dh, a, wb, bb, acc, Po, Pm, fr, 1);
        } else {
            d_pass(Dh, A.Dhoff, wb, acc, Po, 1, 0, pwei, Pm, 1);
        }
    }
    __syncthreads();
    if (part) {
        cd* o = part + (((size_t)zc * nrhs + rhs) * nb + bx) * Ko;
        for (int k = threadIdx.x; k < Ko; k += blockDim.x) o[k] = acc[k];
        continue;
    }
    cd* o = out + (int64_t)rhs * A.ncoef + A.eoff[b];
    for (int k = threadIdx.x; k < Ko; k += blockDim.x) {
        if (mode == 2) o[k] += acc[k];
        else o[k] = acc[k];
    }
    }
}

// sum of the chunk partials of a chunked M2L launch, in chunk order
__global__ void k_tr3h_reduce(const cd* __restrict__ part, int nchunk, int nb, int Ko, int lo,
                              const int64_t* __restrict__ eoff, int64_t ncoef, cd* __restrict__ out) {
    int bi = blockIdx.x, rhs = blockIdx.y, nr = gridDim.y;
    cd* o = out + (int64_t)rhs * ncoef + eoff[lo + bi];
    for (int k = threadIdx.x; k < Ko; k += blockDim.x) {
        cd s = {0, 0};
        for (int z = 0; z < nchunk; ++z) s += part[(((size_t)z * nr + rhs) * nb + bi) * Ko + k];
        o[k] = s;
    }
}

// 3D Laplace translations by the same point-and-shoot scheme (Sec. 5.2,
// Lemma 5.2.4's z-axis forms written for the solid harmonics of fmm3d.cu):
// with U_n^m = Z_n^m / (eps_m s_n^m), T_n^m = eps_m s_n^m Y_n^m / rho^{n+1},
// s_n^m = sqrt((n-|m|)! (n+|m|)!), the Y-basis coefficients of a multipole
// are eps_m s_n^m M_n^m and of a local expansion eps_m L_n^m / s_n^m; the
// rotations of the Helmholtz kernel act on them. Along the z-axis (new centre
// at (0, 0, t) from the old, U_k^0(0,0,z) = z^k/k!, T_j^0(0,0,t) = j!/t^{j+1}):
//   M2M  M'_n^m = sum_k ((-t)^k / k!) M_{n-k}^m
//   M2L  L_k^m  = (-1)^{k+m} sum_n M_n^m (n+k)! / t^{n+k+1}
//   L2L  L'_k^m = sum_{n >= k} L_n^m t^{n-k} / (n-k)!
__global__ void k_tr3l(Tr3hArgs A, int mode, int lo, int P, int d_in_smem, const double* __restrict__ lsm,
                       const double* __restrict__ lsd, const double* __restrict__ fact,
                       const double* __restrict__ ifact, const cd* __restrict__ in, cd* __restrict__ out,
                       int qfirst, const cd* __restrict__ sc, const cd* __restrict__ tt,
                       const int* __restrict__ fb) {
    extern __shared__ cd sm[];
    int b = lo + blockIdx.x;
    if (mode == 0 && A.leaf[b]) return;
    int rhs = blockIdx.y;
    int K = (P + 1) * (P + 1);
    cd* acc = sm;
    cd* a = acc + K;
    cd* bb = a + K;
    cd* wb = bb + K;
    cd* g = wb + K;                     // 2P + 2
    cd* pwe = g + (2 * P + 2);
    cd* pwa = pwe + (2 * P + 1);
    cd* pwai = pwa + (2 * P + 1);
    cd* pwei = pwai + (2 * P + 1);
    double* Dsm = (double*)(pwei + (2 * P + 1));
    const double* Dh = A.Dh;
    if (d_in_smem) {
        int64_t nd = __ldg(A.Dhoff + P + 1);
        for (int64_t k = threadIdx.x; k < nd; k += blockDim.x) Dsm[k] = A.Dh[k];
        Dh = Dsm;
    }
    bool in_local = mode == 2, out_local = mode != 0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) acc[k] = cd{0, 0};
    int qa, qb;
    if (mode == 0) {
        qa = A.cbeg[b];
        qb = A.cend[b];
    } else if (mode == 1) {
        qa = A.loff[b];
        qb = A.loff[b + 1];
    } else {
        qa = 0;
        qb = 1;
    }
    for (int q = qa; q < qb; ++q) {
        int s = mode == 0 ? q : mode == 1 ? A.lent[q] : A.parent[b];
        int p = mode == 2 ? b - lo : q - qfirst;
        __syncthreads();
        const cd* src = in + (int64_t)rhs * A.ncoef + A.eoff[s];
        // Y-basis input
        for (int k = threadIdx.x; k < K; k += blockDim.x) a[k] = (in_local ? __ldg(lsd + k) : __ldg(lsm + k)) * src[k];
        cd t = tt[p];
        int w4 = threadIdx.x >> 5, ln = threadIdx.x & 31;
        if (w4 < 4) {
            cd x = sc[2 * (size_t)p + (w4 >> 1)];
            if (w4 & 1) x = cinv(x);
            cd* dst = (w4 >> 1) ? pwa : pwe;
            for (int m = ln; m <= P; m += 32) dst[P + ((w4 & 1) ? -m : m)] = cpow_int(x, m);
        } else if (w4 == 4) {
            // coaxial factors g[j], j <= 2P+1
            cd base = mode == 0 ? -t : mode == 1 ? cinv(t) : t;
            for (int j = ln; j <= 2 * P + 1; j += 32) {
                cd v = cpow_int(base, mode == 1 ? j + 1 : j);
                g[j] = (mode == 1 ? __ldg(fact + j) : __ldg(ifact + j)) * v;
            }
        }
        __syncthreads();
        for (int m = threadIdx.x - P; m <= P; m += blockDim.x) {
            pwai[P + m] = pwa[P - m];
            pwei[P + m] = pwe[P - m];
        }
        int fr = __ldg(fb + p);
        if (fr >= 0) rot_fixed(A, Dh, a, wb, bb, P, P, fr);
        // forward rotation
        w_pass(A.knm, a, wb, P, 1, 0, pwe, P);
        __syncthreads();
        d_pass(Dh, A.Dhoff, wb, bb, P, 0, 0, nullptr, P, 0);
        __syncthreads();
        w_pass(A.knm, bb, wb, P, 0, 1, pwa, P);
        __syncthreads();
        d_pass(Dh, A.Dhoff, wb, a, P, 1, 0, nullptr, P, 0);
        __syncthreads();
        // back to the solid-harmonic basis, z-axis translation, to the Y basis
        for (int k = threadIdx.x; k < K; k += blockDim.x) a[k] = (in_local ? __ldg(lsm + k) : __ldg(lsd + k)) * a[k];
        __syncthreads();
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            int n, m;
            nm_tab(A.knm, k, n, m);
            int am = m < 0 ? -m : m;
            cd v = {0, 0};
            if (mode == 0) {
                for (int kk = 0; kk <= n - am; ++kk) v = cmac(v, g[kk], a[nmi(n - kk, m)]);
            } else if (mode == 1) {
                for (int nn = am; nn <= P; ++nn) v = cmac(v, g[nn + n], a[nmi(nn, m)]);
                if ((n + m) & 1) v = -v;
            } else {
                for (int nn = n; nn <= P; ++nn) v = cmac(v, g[nn - n], a[nmi(nn, m)]);
            }
            bb[k] = (out_local ? __ldg(lsd + k) : __ldg(lsm + k)) * v;
        }
        __syncthreads();
        // back rotation, accumulated in the solid-harmonic basis
        w_pass(A.knm, bb, wb, P, 1, 0, nullptr, P);
        __syncthreads();
        d_pass(Dh, A.Dhoff, wb, a, P, 0, 0, nullptr, P, 0);
        __syncthreads();
        w_pass(A.knm, a, wb, P, 0, 1, pwai, P);
        __syncthreads();
        d_pass(Dh, A.Dhoff, wb, bb, P, 1, 0, pwei, P, 0);
        __syncthreads();
        if (fr >= 0) {
            rot_fixed_inv(A, Dh, bb, wb, a, bb, P, P, fr, 0);
            __syncthreads();
        }
        for (int k = threadIdx.x; k < K; k += blockDim.x) acc[k] += (out_local ? __ldg(lsm + k) : __ldg(lsd + k)) * bb[k];
    }
    __syncthreads();
    cd* o = out + (int64_t)rhs * A.ncoef + A.eoff[b];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        if (mode == 2) o[k] += acc[k];
        else o[k] = acc[k];
    }
}

// coaxial work arrays of one block (complex entries): sectorial columns and,
// per warp, three recurrence columns and the lower triangle of T^m
size_t tr3h_work(int Pi, int Po, int threads = kH3Threads) {
    int Pn = std::min(Pi, Po), Pm = std::max(Pi, Po), NR = Pi + Po;
    return (size_t)(Pn + 1) * (NR + 1) +
           (size_t)(threads / 32) * ((size_t)3 * (NR + 2) + (size_t)(Pm + 1) * (Pn + 1));
}

size_t tr3h_dh(int P) {
    size_t nd = 0;
    for (int n = 0; n <= P; ++n) nd += (size_t)(n + 1) * (n + 1);
    return nd;
}

size_t tr3h_smem(int Pi, int Po, bool d_in_smem, bool work_in_smem = true, bool acc_in_smem = true,
                 bool flat = false) {
    int Pm = std::max(Pi, Po);
    size_t Km = (size_t)(Pm + 1) * (Pm + 1), Ko = (size_t)(Po + 1) * (Po + 1);
    int NR = Pi + Po;
    size_t work = flat ? (size_t)(Po + 1) * (NR + 1) + tr3h_flat_cols(Po) : tr3h_work(Pi, Po);
    size_t c = (acc_in_smem ? Ko : 0) + 3 * Km + (NR + 1) + 4 * (2 * Pm + 1) + (work_in_smem ? work : 0);
    size_t bytes = c * sizeof(cd);
    if (d_in_smem) bytes += tr3h_dh(Pm) * sizeof(double);
    return bytes;
}

// shared memory of k_tr3h_tri: radial sequence, two column buffers per m,
// triangle offsets
size_t tri_build_smem(int P) {
    return sizeof(cd) * ((size_t)(2 * P + 1) + (size_t)2 * (P + 1) * (2 * P + 2)) + sizeof(int) * (size_t)(P + 1);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Helm3dState {
    int l0 = 1, nlev = 0, maxP = 0;
    std::vector<int> Plev;
    DevBuf<int> dPlev;
    DevBuf<int64_t> exp_off;
    int64_t ncoef = 0;
    std::vector<int> leaves_l0;
    DevBuf<int> d_leaves_l0;
    std::vector<int> p2m_off;    // leaves by level: [p2m_off[l], p2m_off[l+1]) in d_p2m
    DevBuf<int> d_p2m;
    std::vector<int> p2l_off;    // List-4 targets by level, likewise
    int n_p2l = 0;
    DevBuf<int> d_p2l_boxes;
    // single-layer P2M / P2L: per listed box, the offset of its source points in
    // the radial-factor buffer (prefix over the level's boxes)
    DevBuf<int> d_p2m_roff, d_p2l_roff;
    std::vector<int64_t> p2m_rtot, p2l_rtot;    // per level: points in the level's launch
    DevBuf<cd> rad;
    H3Tables* tab = nullptr;
    DevBuf<cd> gscr;             // coaxial work arrays of large-order translations
    DevBuf<cd> part;             // partial results of chunked M2L launches
    std::vector<int> l2max;      // longest List 2 per level
    std::vector<int> l2off;      // host copy of the List-2 offsets
    DevBuf<int> qbox;            // owner box of each List-2 entry
    DevBuf<cd> pre_sc, pre_fl;   // per-pair prologue of a translation launch
    DevBuf<int> pre_fb;          // per pair: fixed frame k, or -1
    DevBuf<cd> pre_pw;           // per pair: e^m, e_a^m for m in [-Pm, Pm]
    DevBuf<cd> tri;              // coaxial operators of the M2L pairs of a launch range
    std::vector<int> level_off;
    int lvl_of_lo(int lo) const {
        for (size_t l = 0; l + 1 < level_off.size(); ++l)
            if (level_off[l] == lo) return (int)l;
        return -1;
    }
};

static std::mutex g_mu;
static std::vector<std::pair<cfmm_plan_s*, Helm3dState*>>& exts() {
    static std::vector<std::pair<cfmm_plan_s*, Helm3dState*>> v;
    return v;
}
static Helm3dState* state(cfmm_plan_s* P) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& e : exts())
        if (e.first == P) return e.second;
    return nullptr;
}
void helm3d_release(cfmm_plan_s* P) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto& v = exts();
    for (size_t i = 0; i < v.size(); ++i)
        if (v[i].first == P) {
            delete v[i].second;
            v.erase(v.begin() + i);
            return;
        }
}

// smallest n with |h_n(kR) j_n(kr)| <= eps for n..n+3 (Eq. nterms_criteria_3d),
// R = (k + 1/2) w, r = sqrt(3)/2 w; a short search first, then up to 2000
static int nterms_helm3d_upto(int k, double eps, double kappa, double w, int pmax) {
    double R = (k + 0.5) * w, r = std::sqrt(3.0) * 0.5 * w;
    std::vector<cd> J(pmax + 4), H(pmax + 4);
    sph_j_seq(cd{kappa * r, 0.0}, pmax + 3, J.data());
    sph_h_seq(cd{kappa * R, 0.0}, pmax + 3, H.data());
    std::vector<char> ok(pmax + 4);
    for (int m = 0; m < pmax + 4; ++m) {
        double a = std::sqrt(cabs2(H[m] * J[m]));
        ok[m] = std::isfinite(a) && a <= eps;
    }
    for (int n = 1; n < pmax; ++n)
        if (ok[n] && ok[n + 1] && ok[n + 2] && ok[n + 3]) return n;
    return -1;
}

int nterms_helm3d(int k, double eps, double kappa, double w) {
    int guess = (int)(kappa * (k + 0.5) * w) + 80;
    if (guess < 2000) {
        int n = nterms_helm3d_upto(k, eps, kappa, w, guess);
        if (n > 0) return n;
    }
    int n = nterms_helm3d_upto(k, eps, kappa, w, 2000);
    return n > 0 ? n : 2000;
}

void helm3d_setup(cfmm_plan_s* P) {
    TreeDev& T = P->tree;
    cudaStream_t st = P->stream;
    Helm3dState* S = new Helm3dState();
    {
        std::lock_guard<std::mutex> lk(g_mu);
        exts().push_back({P, S});
    }
    S->l0 = T.l0;
    S->nlev = T.nlevels;
    S->level_off = T.level_off;
    S->Plev.resize(T.nlevels);
    for (int l = 0; l < T.nlevels; ++l) S->Plev[l] = nterms_helm3d(P->sep, P->eps * 0.01, P->kappa, P->W / (double)(1 << l));
    P->P = S->Plev;
    if (T.nboxes <= 1) return;
    int maxP = 0;
    for (int l = S->l0; l < T.nlevels; ++l) maxP = std::max(maxP, S->Plev[l]);
    CFMM_REQUIRE(maxP <= kH3MaxP, CFMM_EUNSUPPORTED,
                 "3D Helmholtz: expansion order above 63 at the top expansion level (raise top_level or eps)");
    S->maxP = maxP;
    S->tab = tables(maxP);
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
    std::vector<int> lvl(T.nboxes), l4(T.nboxes + 1), l2(T.nboxes + 1), boxes;
    CFMM_CUDA(cudaMemcpyAsync(lvl.data(), T.level.get(), sizeof(int) * T.nboxes, cudaMemcpyDeviceToHost, st));
    CFMM_CUDA(cudaMemcpyAsync(l4.data(), T.loff[3].get(), sizeof(int) * (T.nboxes + 1), cudaMemcpyDeviceToHost, st));
    CFMM_CUDA(cudaMemcpyAsync(l2.data(), T.loff[1].get(), sizeof(int) * (T.nboxes + 1), cudaMemcpyDeviceToHost, st));
    CFMM_CUDA(cudaStreamSynchronize(st));
    S->l2max.assign(T.nlevels, 0);
    for (int b = 0; b < T.nboxes; ++b) S->l2max[lvl[b]] = std::max(S->l2max[lvl[b]], l2[b + 1] - l2[b]);
    S->l2off = l2;
    {
        std::vector<int> qb(std::max(1, l2[T.nboxes]));
        for (int b = 0; b < T.nboxes; ++b)
            for (int q = l2[b]; q < l2[b + 1]; ++q) qb[q] = b;
        S->qbox.alloc(qb.size());
        CFMM_CUDA(cudaMemcpyAsync(S->qbox.get(), qb.data(), sizeof(int) * qb.size(), cudaMemcpyHostToDevice, st));
        CFMM_CUDA(cudaStreamSynchronize(st));
    }
    for (int b : T.leaf_boxes)
        if (lvl[b] >= S->l0) S->leaves_l0.push_back(b);
    S->d_leaves_l0.alloc(S->leaves_l0.size());
    CFMM_CUDA(cudaMemcpyAsync(S->d_leaves_l0.get(), S->leaves_l0.data(), sizeof(int) * S->leaves_l0.size(),
                              cudaMemcpyHostToDevice, st));
    std::vector<int> byl = S->leaves_l0;
    std::stable_sort(byl.begin(), byl.end(), [&](int x, int y) { return lvl[x] < lvl[y]; });
    S->p2m_off.assign(T.nlevels + 1, 0);
    for (int b : byl) S->p2m_off[lvl[b] + 1]++;
    for (int l = 0; l < T.nlevels; ++l) S->p2m_off[l + 1] += S->p2m_off[l];
    S->d_p2m.alloc(byl.size());
    CFMM_CUDA(cudaMemcpyAsync(S->d_p2m.get(), byl.data(), sizeof(int) * byl.size(), cudaMemcpyHostToDevice, st));
    S->p2l_off.assign(T.nlevels + 1, 0);
    for (int b = T.level_off[S->l0]; b < T.nboxes; ++b)
        if (l4[b + 1] > l4[b]) {
            boxes.push_back(b);
            S->p2l_off[lvl[b] + 1]++;
        }
    for (int l = 0; l < T.nlevels; ++l) S->p2l_off[l + 1] += S->p2l_off[l];
    S->n_p2l = (int)boxes.size();
    {
        // radial-buffer offsets of the single-layer P2M / P2L launches
        std::vector<int> hst(T.nboxes), hen(T.nboxes), l4e(std::max(1, l4[T.nboxes]));
        CFMM_CUDA(cudaMemcpyAsync(hst.data(), T.start.get(), sizeof(int) * T.nboxes, cudaMemcpyDeviceToHost, st));
        CFMM_CUDA(cudaMemcpyAsync(hen.data(), T.end.get(), sizeof(int) * T.nboxes, cudaMemcpyDeviceToHost, st));
        if (l4[T.nboxes] > 0)
            CFMM_CUDA(cudaMemcpyAsync(l4e.data(), T.lent[3].get(), sizeof(int) * l4[T.nboxes], cudaMemcpyDeviceToHost,
                                      st));
        CFMM_CUDA(cudaStreamSynchronize(st));
        std::vector<int> ro(byl.size()), rl(boxes.size());
        S->p2m_rtot.assign(T.nlevels, 0);
        S->p2l_rtot.assign(T.nlevels, 0);
        for (int l = 0; l < T.nlevels; ++l) {
            int64_t acc = 0;
            for (int i = S->p2m_off[l]; i < S->p2m_off[l + 1]; ++i) {
                ro[i] = (int)acc;
                acc += hen[byl[i]] - hst[byl[i]];
            }
            S->p2m_rtot[l] = acc;
            acc = 0;
            for (int i = S->p2l_off[l]; i < S->p2l_off[l + 1]; ++i) {
                rl[i] = (int)acc;
                int b = boxes[i];
                for (int q = l4[b]; q < l4[b + 1]; ++q) acc += hen[l4e[q]] - hst[l4e[q]];
            }
            S->p2l_rtot[l] = acc;
        }
        S->d_p2m_roff.alloc(std::max<size_t>(1, ro.size()));
        S->d_p2l_roff.alloc(std::max<size_t>(1, rl.size()));
        if (!ro.empty())
            CFMM_CUDA(cudaMemcpyAsync(S->d_p2m_roff.get(), ro.data(), sizeof(int) * ro.size(), cudaMemcpyHostToDevice, st));
        if (!rl.empty())
            CFMM_CUDA(cudaMemcpyAsync(S->d_p2l_roff.get(), rl.data(), sizeof(int) * rl.size(), cudaMemcpyHostToDevice, st));
    }
    S->d_p2l_boxes.alloc(boxes.size());
    if (!boxes.empty())
        CFMM_CUDA(cudaMemcpyAsync(S->d_p2l_boxes.get(), boxes.data(), sizeof(int) * boxes.size(),
                                  cudaMemcpyHostToDevice, st));
    CFMM_CUDA(cudaStreamSynchronize(st));
    for (auto f : {(const void*)k_p2x3h, (const void*)k_p2x3h_slp<false>, (const void*)k_eval3h, (const void*)k_tr3h,
                   (const void*)k_eval3h_grad, (const void*)k_tr3h_tri})
        CFMM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kH3Smem));
}

void helm3d_apply(cfmm_plan_s* P, const cd* sigma, const cd* tau, int64_t dstride, cd* u, int nrhs, cd* g) {
    Helm3dState* S = state(P);
    CFMM_REQUIRE(S, CFMM_EINVAL, "plan has no 3D Helmholtz state");
    TreeDev& T = P->tree;
    cudaStream_t st = P->stream;
    auto rec = [&](int i) {
        if (P->timing) CFMM_CUDA(cudaEventRecord(P->ev[i], st));
    };
    KParams K{P->xr.get(), P->xi.get(), P->nr.get(), P->ni.get(), P->xr.get(), P->xi.get(), P->n, P->n,
              sigma, tau, dstride, P->slp, P->dlp, P->kappa};
    bool mixed = P->precision == CFMM_MIXED;
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
    H3Tables* TB = S->tab;
    ZCoef zc{TB->zA.get(), TB->zB.get(), TB->dg.get(), TB->s21.get(), TB->knm.get(),
             TB->g3.get(), TB->gp.get(), TB->gm.get()};
    Exp3hArgs A{P->xr.get(), P->xi.get(), P->nr.get(), P->ni.get(), P->n, sigma, tau, dstride, P->slp, P->dlp,
                T.level.get(), T.start.get(), T.end.get(), T.cen_re.get(), T.cen_im.get(), S->dPlev.get(),
                S->exp_off.get(), S->ncoef, P->kappa, zc};
    int maxP = S->maxP;
    // (3) P2P (writes u) on the side stream, beside the far field
    {
        cudaStream_t ns = near_fork(P);
        launch_p2p(3, P->kernel, K, S->d_leaves_l0.get(), (int)S->leaves_l0.size(), T.start.get(), T.end.get(),
                   T.loff[0].get(), T.lent[0].get(), u, nrhs, false, ns, mixed, T.level.get(), P->W, P->sep);
        if (g)
            launch_p2p_grad(3, P->kernel, K, S->d_leaves_l0.get(), (int)S->leaves_l0.size(), T.start.get(),
                            T.end.get(), T.loff[0].get(), T.lent[0].get(), g, nrhs, ns);
    }
    near_launched(P);
    auto p2x_smem = [&](int PL, int& chunk) {
        size_t nc = (size_t)(PL + 1) * (PL + 1);
        size_t per = nc + (PL + 2) + 6;
        chunk = (int)std::max<size_t>(1, std::min<size_t>(32, (96 * 1024 / sizeof(cd) - nc) / per));
        return sizeof(cd) * (nc + (size_t)chunk * per);
    };
    bool slp_only = P->slp && !P->dlp;
    auto slp_fits = [&](int l) {
        size_t K = (size_t)(S->Plev[l] + 1) * (S->Plev[l] + 1);
        return sizeof(cd) * (kH3Threads / 32) * K <= (size_t)kH3Smem;
    };
    // single-layer P2M / P2L of one level: radial factors of every source point,
    // then one warp per source and one lane per harmonic column
    auto p2x_slp = [&](int l, int sing, const int* boxes, int cnt, const int* roff, int64_t rtot, cd* dst) {
        int PL = S->Plev[l];
        S->rad.alloc((size_t)std::max<int64_t>(1, rtot) * (PL + 1));
        k_radial3h<<<cnt, 128, 0, st>>>(A, boxes, cnt, sing ? T.loff[3].get() : nullptr,
                                         sing ? T.lent[3].get() : nullptr, sing, PL, roff, S->rad.get());
        CFMM_LAUNCHED();
        size_t smem = sizeof(cd) * (size_t)(kH3Threads / 32) * (PL + 1) * (PL + 1);
        dim3 g((unsigned)cnt, nrhs);
        k_p2x3h_slp<false><<<g, kH3Threads, smem, st>>>(A, boxes, sing ? T.loff[3].get() : nullptr,
                                                        sing ? T.lent[3].get() : nullptr, sing, roff, S->rad.get(),
                                                        dst, nullptr);
        CFMM_LAUNCHED();
    };
    // (1) P2M, one launch per level (shared memory sized by that level's P)
    for (int l = S->l0; l < T.nlevels; ++l) {
        int cnt = S->p2m_off[l + 1] - S->p2m_off[l];
        if (cnt <= 0) continue;
        if (slp_only && mixed && p2m3f_smem(S->Plev[l]) <= (size_t)kH3Smem) {
            // complex64 products, FP64 sums
            launch_p2m3f(TB, true, P, S->d_p2m.get() + S->p2m_off[l], cnt, S->Plev[l], S->dPlev.get(),
                         S->exp_off.get(), S->ncoef, sigma, dstride, mp, nrhs);
            continue;
        }
        if (slp_only && slp_fits(l)) {
            p2x_slp(l, 0, S->d_p2m.get() + S->p2m_off[l], cnt, S->d_p2m_roff.get() + S->p2m_off[l], S->p2m_rtot[l], mp);
            continue;
        }
        int chunk;
        size_t smem = p2x_smem(S->Plev[l], chunk);
        dim3 g((unsigned)cnt, nrhs);
        k_p2x3h<<<g, kH3Threads, smem, st>>>(A, S->d_p2m.get() + S->p2m_off[l], nullptr, nullptr, 0, mp, chunk);
        CFMM_LAUNCHED();
    }
    rec(2);
    Tr3hArgs TA{T.cen_re.get(), T.cen_im.get(), S->exp_off.get(), S->ncoef, TB->Dh.get(), TB->Dhoff.get(),
                TB->inv2n1.get(), TB->al.get(), TB->be.get(), TB->ibe.get(), TB->mu.get(), TB->nu.get(),
                TB->knm.get(), P->kappa, T.cbeg.get(), T.cend.get(),
                T.loff[1].get(), T.lent[1].get(), T.parent.get(), T.leaf.get(), S->qbox.get()};
    int nsm = 0;
    CFMM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P->device));
    auto launch_range = [&](int mode, int lo, int nb, int Pi, int Po, int use_h, const cd* in, cd* out, int nchunk,
                            int chunk, bool tri) {
        if (nb <= 0) return;
        // the flat coaxial work (equal orders, everything in shared memory with
        // the rotation table) for the translations of the lower levels
        int flat = (!tri && Pi == Po && Pi <= kTr3FlatMaxP &&
                    tr3h_smem(Pi, Po, true, true, true, true) <= (size_t)kH3Smem) ? 1 : 0;
        size_t smem = tri ? tr3h_smem(Pi, Po, true, false) : tr3h_smem(Pi, Po, true, true, true, flat != 0);
        int dsm = 1;
        cd* gs = nullptr;
        if (smem > (size_t)kH3Smem) {
            smem = tr3h_smem(Pi, Po, false, !tri);
            dsm = 0;
        }
        int64_t nitem = (int64_t)nb * nrhs * nchunk, G = nitem;
        int accg = 0, threads = kH3Threads;
        if (!tri && smem > (size_t)kH3Smem) {
            // coaxial work arrays (and for the largest orders the accumulator)
            // in global scratch: one slice per resident block, the blocks
            // stride over the work items
            smem = tr3h_smem(Pi, Po, false, false);
            if (smem > (size_t)kH3Smem) {
                // one block per SM fits: twice the threads keep the FP64 pipe fed
                smem = tr3h_smem(Pi, Po, false, false, false);
                accg = 1;
                threads = 2 * kH3Threads;
            }
            int per_sm = 0;
            CFMM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tr3h, threads, smem));
            G = std::min<int64_t>(nitem, (int64_t)std::max(1, per_sm) * nsm);
            size_t per = tr3h_work(Pi, Po, threads) + (accg ? (size_t)(Po + 1) * (Po + 1) : 0);
            S->gscr.alloc(per * (size_t)G);
            gs = S->gscr.get();
        }
        CFMM_REQUIRE(smem <= (size_t)kH3Smem, CFMM_EUNSUPPORTED, "3D Helmholtz translation exceeds shared memory");
        dim3 g((unsigned)G);
        size_t Ko = (size_t)(Po + 1) * (Po + 1);
        cd* pp = nullptr;
        if (nchunk > 1) {
            S->part.alloc(Ko * nb * nrhs * nchunk);
            pp = S->part.get();
        }
        // per-pair prologue (shift, rotation scalars, radial sequence)
        int qfirst, npair;
        if (mode == 1) {
            qfirst = S->l2off[lo];
            npair = S->l2off[lo + nb] - qfirst;
        } else if (mode == 0) {
            int l = S->lvl_of_lo(lo);
            qfirst = T.level_off[l + 1];
            npair = T.level_off[l + 2] - qfirst;
        } else {
            qfirst = lo;
            npair = nb;
        }
        int NR = Pi + Po;
        S->pre_sc.alloc((size_t)2 * std::max(npair, 1));
        S->pre_fl.alloc((size_t)(NR + 1) * std::max(npair, 1));
        S->pre_fb.alloc((size_t)std::max(npair, 1));
        int Pmx = std::max(Pi, Po);
        S->pre_pw.alloc((size_t)2 * (2 * Pmx + 1) * std::max(npair, 1));
        if (npair > 0) {
            k_tr3h_pre<<<(npair + 127) / 128, 128, 0, st>>>(TA, mode, lo, qfirst, npair, NR, use_h, S->pre_sc.get(),
                                                           S->pre_fl.get(), S->pre_fb.get(), Pmx, S->pre_pw.get());
            CFMM_LAUNCHED();
        }
        const cd* trig = nullptr;
        if (tri && npair > 0) {
            S->tri.alloc(tr3h_tri_size(Pi) * (size_t)npair);
            k_tr3h_tri<<<npair, kTriThreads, tri_build_smem(Pi), st>>>(TA, Pi, npair, S->pre_fl.get(), S->tri.get());
            CFMM_LAUNCHED();
            trig = S->tri.get();
        }
        k_tr3h<<<g, threads, smem, st>>>(TA, mode, lo, nb, Pi, Po, use_h, dsm, gs, in, out, chunk, pp,
                                            qfirst, S->pre_pw.get(), S->pre_fl.get(), nrhs, nchunk, accg, flat,
                                            S->pre_fb.get(), tri ? 1 : 0, trig);
        CFMM_LAUNCHED();
        if (nchunk > 1) {
            k_tr3h_reduce<<<dim3(nb, nrhs), 256, 0, st>>>(pp, nchunk, nb, (int)Ko, lo, S->exp_off.get(), S->ncoef,
                                                          out);
            CFMM_LAUNCHED();
        }
    };
    auto launch_tr = [&](int mode, int lo, int nb, int Pi, int Po, int use_h, const cd* in, cd* out, int nchunk,
                         int chunk) {
        // M2L at equal orders up to kTriMaxP (kTriMaxPMulti with several
        // right-hand sides): the coaxial operators of the level's pairs are
        // built first by k_tr3h_tri (in HBM, once for every right-hand side),
        // over box ranges whose operators fit kTriBudget
        bool tri = mode == 1 && Pi == Po && (Pi <= kTriMaxP || (nrhs > 1 && Pi <= kTriMaxPMulti)) &&
                   tri_build_smem(Pi) <= (size_t)kH3Smem && tr3h_smem(Pi, Po, false, false) <= (size_t)kH3Smem;
        if (!tri) {
            launch_range(mode, lo, nb, Pi, Po, use_h, in, out, nchunk, chunk, false);
            return;
        }
        int64_t cap = std::max<int64_t>(1, (int64_t)(kTriBudget / (tr3h_tri_size(Pi) * sizeof(cd))));
        for (int b0 = lo; b0 < lo + nb;) {
            int b1 = b0 + 1;
            while (b1 < lo + nb && S->l2off[b1 + 1] - S->l2off[b0] <= cap) ++b1;
            launch_range(mode, b0, b1 - b0, Pi, Po, use_h, in, out, nchunk, chunk, true);
            b0 = b1;
        }
    };
    // (2) M2M: parents at level l from children at l + 1 (leaf parents get zeros
    // from an empty child range)
    for (int l = T.nlevels - 2; l >= S->l0; --l) {
        int lo = T.level_off[l], nb = T.level_off[l + 1] - lo;
        launch_tr(0, lo, nb, S->Plev[l + 1], S->Plev[l], 0, mp, mp, 1, 1);
    }
    rec(3);
    // (4) M2L per level (overwrites L at levels >= l0)
    for (int l = S->l0; l < T.nlevels; ++l) {
        int lo = T.level_off[l], nb = T.level_off[l + 1] - lo;
        // long lists (the all-pairs top level) are split over several blocks,
        // as far as the launch needs more blocks (many right-hand sides already
        // give enough, and then no partials are written)
        int nchunk = S->l2max[l] > 2 * kM2LChunk3 ? (S->l2max[l] + kM2LChunk3 - 1) / kM2LChunk3 : 1;
        int64_t want = (int64_t)16 * nsm, base = (int64_t)std::max(1, nb) * nrhs;
        if (nchunk > 1 && base * nchunk > want) nchunk = (int)std::max<int64_t>(1, (want + base - 1) / base);
        // few boxes (a coarse top level): split their lists down to 4 entries
        // so that every SM gets work
        if (base * nchunk < want && S->l2max[l] > 4)
            nchunk = (int)std::max<int64_t>(nchunk, std::min<int64_t>((S->l2max[l] + 3) / 4, (want + base - 1) / base));
        int chunk = nchunk > 1 ? (S->l2max[l] + nchunk - 1) / nchunk : std::max(1, S->l2max[l]);
        launch_tr(1, lo, nb, S->Plev[l], S->Plev[l], 1, mp, lc, nchunk, chunk);
    }
    rec(4);
    // (6) P2L, per level
    for (int l = S->l0; l < T.nlevels; ++l) {
        int cnt = S->p2l_off[l + 1] - S->p2l_off[l];
        if (cnt <= 0) continue;
        if (slp_only && slp_fits(l)) {
            p2x_slp(l, 1, S->d_p2l_boxes.get() + S->p2l_off[l], cnt, S->d_p2l_roff.get() + S->p2l_off[l],
                    S->p2l_rtot[l], lc);
            continue;
        }
        int chunk;
        size_t smem = p2x_smem(S->Plev[l], chunk);
        dim3 g((unsigned)cnt, nrhs);
        k_p2x3h<<<g, kH3Threads, smem, st>>>(A, S->d_p2l_boxes.get() + S->p2l_off[l], T.loff[3].get(),
                                             T.lent[3].get(), 1, lc, chunk);
        CFMM_LAUNCHED();
    }
    rec(5);
    // (7) L2L
    for (int l = S->l0 + 1; l < T.nlevels; ++l) {
        int lo = T.level_off[l], nb = T.level_off[l + 1] - lo;
        launch_tr(2, lo, nb, S->Plev[l - 1], S->Plev[l], 0, lc, lc, 1, 1);
    }
    rec(6);
    rec(7);
    near_join(P);   // the near field has written u
    // (5) M2P, (8) L2P (complex64 in mixed precision)
    {
        dim3 gr((unsigned)S->leaves_l0.size(), nrhs);
        k_eval3h<<<gr, 128, sizeof(cd) * (size_t)(maxP + 1) * (maxP + 1), st>>>(
            A, S->d_leaves_l0.get(), T.loff[2].get(), T.lent[2].get(), mp, lc, u, mixed ? 0 : 1);
        CFMM_LAUNCHED();
        if (mixed) launch_l2p3f(TB, true, P, S->d_leaves_l0.get(), (int)S->leaves_l0.size(), maxP, S->dPlev.get(),
                                S->exp_off.get(), S->ncoef, lc, u, nrhs);
        if (g && gr.x) {
            k_eval3h_grad<<<gr, 128, sizeof(cd) * (size_t)(maxP + 1) * (maxP + 1), st>>>(
                A, S->d_leaves_l0.get(), T.loff[2].get(), T.lent[2].get(), mp, lc, g);
            CFMM_LAUNCHED();
        }
    }
    rec(8);
}

// ---------------------------------------------------------------------------
// 3D Laplace translations through k_tr3l (used by fmm3d.cu)
// ---------------------------------------------------------------------------
struct Lap3Tr {
    H3Tables* tab = nullptr;
    int Pord = 0;
    std::vector<int> l2off, level_off;
    DevBuf<int> qbox;
    DevBuf<cd> sc, tt;
    DevBuf<int> fb;
};

Lap3Tr* lap3_tr_create(cfmm_plan_s* P, int Pord) {
    TreeDev& T = P->tree;
    cudaStream_t st = P->stream;
    Lap3Tr* L = new Lap3Tr();
    L->tab = tables(Pord);
    L->level_off = T.level_off;
    L->l2off.resize(T.nboxes + 1);
    CFMM_CUDA(cudaMemcpyAsync(L->l2off.data(), T.loff[1].get(), sizeof(int) * (T.nboxes + 1), cudaMemcpyDeviceToHost,
                              st));
    CFMM_CUDA(cudaStreamSynchronize(st));
    std::vector<int> qb(std::max(1, L->l2off[T.nboxes]));
    for (int b = 0; b < T.nboxes; ++b)
        for (int q = L->l2off[b]; q < L->l2off[b + 1]; ++q) qb[q] = b;
    L->qbox.alloc(qb.size());
    CFMM_CUDA(cudaMemcpyAsync(L->qbox.get(), qb.data(), sizeof(int) * qb.size(), cudaMemcpyHostToDevice, st));
    CFMM_CUDA(cudaStreamSynchronize(st));
    CFMM_CUDA(cudaFuncSetAttribute((const void*)k_tr3l, cudaFuncAttributeMaxDynamicSharedMemorySize, kH3Smem));
    CFMM_CUDA(cudaFuncSetAttribute((const void*)k_p2x3h_slp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kH3Smem));
    L->Pord = Pord;
    return L;
}

bool lap3_p2m_slp(Lap3Tr* L, cfmm_plan_s* P, const int* leaves, int cnt, int maxP, const int* dPlev,
                  const int64_t* eoff, int64_t ncoef, const cd* sigma, int64_t dstride, cd* out, int nrhs) {
    size_t smem = sizeof(cd) * (size_t)(kH3Threads / 32) * (maxP + 1) * (maxP + 1);
    if (smem > (size_t)kH3Smem || maxP > L->Pord) return false;
    if (cnt <= 0) return true;
    TreeDev& T = P->tree;
    H3Tables* TB = L->tab;
    ZCoef zc{TB->zA.get(), TB->zB.get(), TB->dg.get(), TB->s21.get(), TB->knm.get(),
             TB->g3.get(), TB->gp.get(), TB->gm.get()};
    Exp3hArgs A{P->xr.get(), P->xi.get(), nullptr, nullptr, P->n, sigma, nullptr, dstride, true, false,
                T.level.get(), T.start.get(), T.end.get(), T.cen_re.get(), T.cen_im.get(), dPlev, eoff, ncoef,
                0.0, zc};
    dim3 g((unsigned)cnt, nrhs);
    k_p2x3h_slp<true><<<g, kH3Threads, smem, P->stream>>>(A, leaves, nullptr, nullptr, 0, nullptr, nullptr, out,
                                                          TB->lsd.get());
    CFMM_LAUNCHED();
    return true;
}

bool lap3_p2m32(Lap3Tr* L, cfmm_plan_s* P, const int* leaves, int cnt, int maxP, const int* dPlev,
                const int64_t* eoff, int64_t ncoef, const cd* sigma, int64_t dstride, cd* out, int nrhs) {
    if (maxP > L->tab->Pmax || p2m3f_smem(maxP) > (size_t)kH3Smem) return false;
    launch_p2m3f(L->tab, false, P, leaves, cnt, maxP, dPlev, eoff, ncoef, sigma, dstride, out, nrhs);
    return true;
}

void lap3_l2p32(Lap3Tr* L, cfmm_plan_s* P, const int* leaves, int cnt, int maxP, const int* dPlev,
                const int64_t* eoff, int64_t ncoef, const cd* loc, cd* u, int nrhs) {
    CFMM_REQUIRE(maxP <= L->tab->Pmax, CFMM_ECUDA, "3D Laplace L2P: order beyond the tables");
    launch_l2p3f(L->tab, false, P, leaves, cnt, maxP, dPlev, eoff, ncoef, loc, u, nrhs);
}

void lap3_tr_destroy(Lap3Tr* L) { delete L; }

// mode 0: M2M into the non-leaf boxes of level l from level l+1; 1: M2L at
// level l (writes L); 2: L2L into level l from level l-1 (adds)
void lap3_tr_launch(Lap3Tr* L, cfmm_plan_s* P, int mode, int l, int Pord, const int64_t* eoff, int64_t ncoef,
                    const cd* in, cd* out, int nrhs) {
    TreeDev& T = P->tree;
    cudaStream_t st = P->stream;
    int lo = T.level_off[l], nb = T.level_off[l + 1] - lo;
    if (nb <= 0) return;
    H3Tables* TB = L->tab;
    Tr3hArgs TA{T.cen_re.get(), T.cen_im.get(), eoff, ncoef, TB->Dh.get(), TB->Dhoff.get(),
                TB->inv2n1.get(), TB->al.get(), TB->be.get(), TB->ibe.get(), TB->mu.get(), TB->nu.get(),
                TB->knm.get(), 0.0, T.cbeg.get(), T.cend.get(), T.loff[1].get(), T.lent[1].get(), T.parent.get(),
                T.leaf.get(), L->qbox.get()};
    int qfirst, npair;
    if (mode == 1) {
        qfirst = L->l2off[lo];
        npair = L->l2off[lo + nb] - qfirst;
    } else if (mode == 0) {
        qfirst = T.level_off[l + 1];
        npair = T.level_off[l + 2] - qfirst;
    } else {
        qfirst = lo;
        npair = nb;
    }
    L->sc.alloc((size_t)2 * std::max(npair, 1));
    L->tt.alloc((size_t)std::max(npair, 1));
    L->fb.alloc((size_t)std::max(npair, 1));
    if (npair > 0) {
        k_tr3h_pre<<<(npair + 127) / 128, 128, 0, st>>>(TA, mode, lo, qfirst, npair, -1, 0, L->sc.get(), L->tt.get(),
                                                       L->fb.get(), 0, nullptr);
        CFMM_LAUNCHED();
    }
    size_t K = (size_t)(Pord + 1) * (Pord + 1);
    size_t smem = sizeof(cd) * (4 * K + (2 * Pord + 2) + 4 * (2 * Pord + 1));
    size_t nd = tr3h_dh(Pord) * sizeof(double);
    int dsm = smem + nd <= (size_t)kH3Smem;
    if (dsm) smem += nd;
    CFMM_REQUIRE(smem <= (size_t)kH3Smem, CFMM_EUNSUPPORTED, "3D Laplace translation exceeds shared memory");
    dim3 g(nb, nrhs);
    k_tr3l<<<g, kH3Threads, smem, st>>>(TA, mode, lo, Pord, dsm, TB->lsm.get(), TB->lsd.get(), TB->fact.get(),
                                        TB->ifact.get(), in, out, qfirst, L->sc.get(), L->tt.get(), L->fb.get());
    CFMM_LAUNCHED();
}

}  // namespace cfmm
