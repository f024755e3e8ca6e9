// Complex special functions for the CUDA path (host and device).
//
// Everything is built from sqrt, log, exp, sin/cos and atan2 calls plus the
// series, recurrences and quadratures named below:
//   * principal complex sqrt / log (branch cut on the negative real axis);
//   * H_0^(1), H_1^(1) of complex z with Re z > 0:
//       |z| <= 6 : ascending series for J_0, J_1, Y_0, Y_1 (DLMF 10.2.2, 10.8.1);
//       |z| >  6 : the Laplace-type integral
//                  H_nu(z) = sqrt(2/(pi z)) e^{i(z - nu pi/2 - pi/4)} / Gamma(nu+1/2)
//                            * int_0^inf e^{-u} u^{nu-1/2} (1 + iu/(2z))^{nu-1/2} du
//                  (Watson, Treatise, Sec. 7.2; the integral behind the
//                  expansion DLMF 10.17.5) by 24-point generalized
//                  Gauss-Laguerre quadrature (alpha = -1/2, +1/2);
//   * J_0..J_n of complex z by Miller's backward recurrence (DLMF 10.74(iv)),
//     normalised with exp(-/+ i z) = J_0 + 2 sum (-/+ i)^k J_k (generating
//     function DLMF 10.12.1 at t = -/+ i), the sign chosen so the sum does
//     not cancel;
//   * H_n by forward recurrence H_{n+1} = (2n/z) H_n - H_{n-1} (DLMF 10.6.1);
//   * spherical h_n^(1)(z) from h_0 = -i e^{iz}/z, h_1 = -e^{iz}(z + i)/z^2
//     and forward recurrence h_{n+1} = ((2n+1)/z) h_n - h_{n-1} (DLMF 10.49.6,
//     10.51.1; h_n is the dominant solution);
//   * spherical j_n(z) by Miller's backward recurrence, normalised with
//     exp(-/+ i z) = sum (2n+1) (-/+ i)^n j_n(z) (the plane-wave expansion
//     DLMF 10.60.7 at cos = -/+ 1), the sign chosen so the sum does not cancel.
#pragma once

#include "cfmm_common.cuh"

namespace cfmm {

// Every translation unit that includes this header owns a copy of the rule in
// its constant bank; the TU's own upload function (declared below) fills it.
static __constant__ LagRule c_lag;
static inline void upload_lag_rule_local() {
    CFMM_CUDA(cudaMemcpyToSymbol(c_lag, &host_lag_rule(), sizeof(LagRule)));
}

CFMM_HD cd csqrt_p(cd z) {
    double a = z.x, b = z.y;
    if (a == 0.0 && b == 0.0) return cd{0.0, 0.0};
    double m = hypot(a, b);
    double t = sqrt(0.5 * (fabs(a) + m));
    if (a >= 0.0) return cd{t, b / (2.0 * t)};
    return cd{fabs(b) / (2.0 * t), copysign(t, b)};
}

CFMM_HD cd clog_p(cd z) { return cd{log(hypot(z.x, z.y)), atan2(z.y, z.x)}; }

CFMM_HD cd cexp_p(cd z) {
    double e = exp(z.x), s, c;
    sincos(z.y, &s, &c);
    return cd{e * c, e * s};
}

// e^{i z} for complex z
CFMM_HD cd cexp_i(cd z) { return cexp_p(cd{-z.y, z.x}); }

// H_0^(1)(z), H_1^(1)(z) for complex z, Re z >= 0 (|arg z| < pi/2).
CFMM_HD void hankel01(cd z, cd* h0, cd* h1) {
    const double kPi = 3.14159265358979323846;
    const double kEulerGamma = 0.57721566490153286061;
    double az = hypot(z.x, z.y);
    if (az <= kHankelSeriesMax) {
        cd q = 0.25 * (z * z);
        cd mq = -q;
        // J0 = sum t_k, t_k = (-q)^k/(k!)^2 ; Y0 sum: -sum_{k>=1} H_k t_k
        // J1 = (z/2) sum s_k, s_k = (-q)^k/(k!(k+1)!)
        // Y1 sum: sum_k (psi(k+1)+psi(k+2)) s_k,  psi(k+1) = -gamma + H_k
        cd t = {1.0, 0.0}, s = {1.0, 0.0};
        cd j0 = t, j1s = s, y0s = {0.0, 0.0};
        cd y1s = (-2.0 * kEulerGamma + 1.0) * s;   // k=0: psi(1)+psi(2) = -2gamma + 1
        double Hk = 0.0;
        for (int k = 1; k < 60; ++k) {
            double dk = (double)k;
            t = t * mq * (1.0 / (dk * dk));
            s = s * mq * (1.0 / (dk * (dk + 1.0)));
            Hk += 1.0 / dk;
            j0 += t;
            j1s += s;
            y0s -= Hk * t;
            y1s += (-2.0 * kEulerGamma + 2.0 * Hk + 1.0 / (dk + 1.0)) * s;
            if (cabs2(t) < 1e-40 && cabs2(s) < 1e-40) break;
        }
        cd zh = 0.5 * z;
        cd lz = clog_p(zh);
        cd j1 = zh * j1s;
        cd y0 = (2.0 / kPi) * ((lz + cd{kEulerGamma, 0.0}) * j0 + y0s);
        cd y1 = (-2.0 / kPi) * cinv(z) + (2.0 / kPi) * (lz * j1) - (1.0 / kPi) * (zh * y1s);
        *h0 = j0 + mul_i(y0);
        *h1 = j1 + mul_i(y1);
        return;
    }
#ifdef __CUDA_ARCH__
    const LagRule& L = c_lag;
#else
    const LagRule& L = host_lag_rule();
#endif
    cd a = mul_i(cinv(2.0 * z));   // i/(2z)
    cd s0 = {0.0, 0.0}, s1 = {0.0, 0.0};
#pragma unroll 4
    for (int i = 0; i < kLagNodes; ++i) {
        cd q0 = cd{1.0, 0.0} + L.x[0][i] * a;
        cd q1 = cd{1.0, 0.0} + L.x[1][i] * a;
        s0 += L.w[0][i] * cinv(csqrt_p(q0));
        s1 += L.w[1][i] * csqrt_p(q1);
    }
    // sqrt(2/(pi z)) e^{i(z - pi/4)} / Gamma(1/2);  Gamma(1/2)=sqrt(pi), Gamma(3/2)=sqrt(pi)/2
    cd pre = sqrt(2.0 / kPi) * cinv(csqrt_p(z));
    cd ez = cexp_i(z);
    const double r2 = 0.70710678118654752440;
    cd e0 = ez * cd{r2, -r2};          // e^{i(z - pi/4)}
    cd e1 = ez * cd{-r2, -r2};         // e^{i(z - 3pi/4)}
    const double isp = 0.56418958354775628695;   // 1/sqrt(pi)
    *h0 = (isp * pre) * e0 * s0;
    *h1 = (2.0 * isp * pre) * e1 * s1;
}

// J_0..J_nmax of complex z (Miller, normalised as described above).
// out must hold nmax+1 values.
CFMM_HD void bessel_j_seq(cd z, int nmax, cd* out) {
    double az = hypot(z.x, z.y);
    if (az == 0.0) {
        out[0] = cd{1.0, 0.0};
        for (int n = 1; n <= nmax; ++n) out[n] = cd{0.0, 0.0};
        return;
    }
    double big = az > (double)nmax ? az : (double)nmax;
    // start index: a short start for |z| <= 2 (the terms beyond nmax fall off
    // like (|z|/2)^k / k!; 12 + 4|z| extra orders agree with the long start to
    // 4e-15 relative, checked for nmax <= 60), the long one otherwise
    int N0 = az <= 2.0 ? nmax + 13 + (int)(4.0 * az) : (int)big + 24 + (int)sqrt(32.0 * big);
    bool up = z.y >= 0.0;                  // use exp(-iz) = sum (-i)^k eps_k J_k
    cd zi = cinv(z);
    cd fp = {0.0, 0.0}, f = {1e-200, 0.0};
    cd S = {0.0, 0.0};
    for (int n = 0; n <= nmax; ++n) out[n] = cd{0.0, 0.0};
    for (int n = N0; n >= 1; --n) {
        if (n <= nmax) out[n] = f;
        // (-i)^n or i^n times 2 f
        cd w;
        int r = n & 3;
        if (up) w = (r == 0) ? f : (r == 1) ? cd{f.y, -f.x} : (r == 2) ? -f : cd{-f.y, f.x};
        else    w = (r == 0) ? f : (r == 1) ? cd{-f.y, f.x} : (r == 2) ? -f : cd{f.y, -f.x};
        S = cd{fma(2.0, w.x, S.x), fma(2.0, w.y, S.y)};
        cd t = zi * f;
        cd fm = {fma(2.0 * n, t.x, -fp.x), fma(2.0 * n, t.y, -fp.y)};
        fp = f;
        f = fm;
        if (cabs2(f) > 1e300) {
            const double sc = 1e-150;
            f = sc * f;
            fp = sc * fp;
            S = sc * S;
            int top = nmax < N0 ? nmax : N0;
            for (int m = n; m <= top; ++m) out[m] = sc * out[m];
        }
    }
    out[0] = f;
    S += f;
    cd e = up ? cexp_i(-z) : cexp_i(z);
    cd scale = e / S;
    for (int n = 0; n <= nmax; ++n) out[n] = out[n] * scale;
}

// h_n^(1)(z), n = 0..nmax, complex z != 0
CFMM_HD void sph_h_seq(cd z, int nmax, cd* out) {
    cd e = cexp_i(z);
    cd zi = cinv(z);
    out[0] = -mul_i(e * zi);
    if (nmax < 1) return;
    out[1] = -(e * (z + cd{0.0, 1.0})) * (zi * zi);
    for (int n = 1; n < nmax; ++n) out[n + 1] = rmac(-out[n - 1], 2.0 * n + 1.0, zi * out[n]);
}

// j_n(z), n = 0..nmax, complex z
CFMM_HD void sph_j_seq(cd z, int nmax, cd* out) {
    double az = hypot(z.x, z.y);
    if (az == 0.0) {
        out[0] = cd{1.0, 0.0};
        for (int n = 1; n <= nmax; ++n) out[n] = cd{0.0, 0.0};
        return;
    }
    double big = az > (double)nmax ? az : (double)nmax;
    // short start for |z| <= 2 as in bessel_j_seq (agrees to 5e-15, nmax <= 80)
    int N0 = az <= 2.0 ? nmax + 13 + (int)(4.0 * az) : (int)big + 24 + (int)sqrt(32.0 * big);
    bool up = z.y >= 0.0;                  // exp(-iz) = sum (2n+1) (-i)^n j_n
    cd zi = cinv(z);
    cd fp = {0.0, 0.0}, f = {1e-200, 0.0};
    cd S = {0.0, 0.0};
    for (int n = 0; n <= nmax; ++n) out[n] = cd{0.0, 0.0};
    for (int n = N0; n >= 1; --n) {
        if (n <= nmax) out[n] = f;
        cd w;
        int r = n & 3;
        if (up) w = (r == 0) ? f : (r == 1) ? cd{f.y, -f.x} : (r == 2) ? -f : cd{-f.y, f.x};
        else    w = (r == 0) ? f : (r == 1) ? cd{-f.y, f.x} : (r == 2) ? -f : cd{f.y, -f.x};
        double c2 = 2.0 * n + 1.0;
        S = cd{fma(c2, w.x, S.x), fma(c2, w.y, S.y)};
        cd t = zi * f;
        cd fm = {fma(c2, t.x, -fp.x), fma(c2, t.y, -fp.y)};   // j_{n-1} = ((2n+1)/z) j_n - j_{n+1}
        fp = f;
        f = fm;
        if (cabs2(f) > 1e300) {
            const double sc = 1e-150;
            f = sc * f;
            fp = sc * fp;
            S = sc * S;
            int top = nmax < N0 ? nmax : N0;
            for (int m = n; m <= top; ++m) out[m] = sc * out[m];
        }
    }
    out[0] = f;
    S += f;
    cd e = up ? cexp_i(-z) : cexp_i(z);
    cd scale = e / S;
    for (int n = 0; n <= nmax; ++n) out[n] = out[n] * scale;
}

}  // namespace cfmm
