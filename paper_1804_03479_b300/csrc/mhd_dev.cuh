// mhd_dev.cuh -- device-side physics of the MHD patch advance (sm_103a).
//
// Everything here works on the 1-D "sweep frame" of one axis n with the two
// transverse axes t1 = n+1, t2 = n+2 (cyclic):
//   w = (rho, v_n, v_t1, v_t2, P, B_t1, B_t2),  B_n carried separately,
//   flux / conserved order (rho, M_n, M_t1, M_t2, e, B_t1, B_t2).
// Templated on the arithmetic type R (double or float).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace mhd {

enum { VL = 0, CTU = 1 };
enum { PLM = 0, PPM = 1, PLM_PRIM = 2 };
enum { ROE = 0, HLLD = 1, HLLE = 2 };

template <class R> struct Num;
template <> struct Num<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
    static __device__ __forceinline__ double abs_(double x) { return fabs(x); }
    static __device__ __forceinline__ double min_(double a, double b) { return fmin(a, b); }
    static __device__ __forceinline__ double max_(double a, double b) { return fmax(a, b); }
    static __device__ __forceinline__ double copysign_(double a, double b) { return copysign(a, b); }
    static constexpr double hlld_degen = 1e-8;
    static constexpr double fan_margin = 1e-10;   // relative margin of the Roe fan bound
};
template <> struct Num<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float abs_(float x) { return fabsf(x); }
    static __device__ __forceinline__ float min_(float a, float b) { return fminf(a, b); }
    static __device__ __forceinline__ float max_(float a, float b) { return fmaxf(a, b); }
    static __device__ __forceinline__ float copysign_(float a, float b) { return copysignf(a, b); }
    static constexpr float hlld_degen = 1e-5f;
    static constexpr float fan_margin = 1e-4f;
};

// one min/max instruction each; for ordered operands the value of a < b ? a : b
// (at most the sign of a zero result differs)
template <class R> __device__ __forceinline__ R rmin(R a, R b) { return Num<R>::min_(a, b); }
template <class R> __device__ __forceinline__ R rmax(R a, R b) { return Num<R>::max_(a, b); }
template <class R> __device__ __forceinline__ R sgn1(R a) { return a >= R(0) ? R(1) : R(-1); }

// ---- Eq. 5 and Eqs. 7-9 in the sweep frame ------------------------------
template <class R>
__device__ __forceinline__ R total_energy(const R w[7], R bn, R gm1)
{
    R v2 = w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
    R b2 = bn * bn + w[5] * w[5] + w[6] * w[6];
    return w[4] / gm1 + R(0.5) * w[0] * v2 + R(0.5) * b2;
}

template <class R>
__device__ __forceinline__ void to_cons(const R w[7], R bn, R gm1, R u[7])
{
    u[0] = w[0];
    u[1] = w[0] * w[1];
    u[2] = w[0] * w[2];
    u[3] = w[0] * w[3];
    u[4] = total_energy(w, bn, gm1);
    u[5] = w[5];
    u[6] = w[6];
}

template <class R>
__device__ __forceinline__ void phys_flux(const R w[7], R bn, R gm1, R f[7])
{
    R e = total_energy(w, bn, gm1);
    R pt = w[4] + R(0.5) * (bn * bn + w[5] * w[5] + w[6] * w[6]);
    R vb = w[1] * bn + w[2] * w[5] + w[3] * w[6];
    f[0] = w[0] * w[1];
    f[1] = w[0] * w[1] * w[1] + pt - bn * bn;
    f[2] = w[0] * w[1] * w[2] - bn * w[5];
    f[3] = w[0] * w[1] * w[3] - bn * w[6];
    f[4] = (e + pt) * w[1] - bn * vb;
    f[5] = w[5] * w[1] - bn * w[2];
    f[6] = w[6] * w[1] - bn * w[3];
}

// fast magnetosonic speed; FP32 multiplies by 1/rho (one reciprocal serves
// both field terms), FP64 divides by rho as the oracle does
template <class R>
__device__ __forceinline__ R fast_speed(R rho, R irho, R a2, R bn, R bt1, R bt2)
{
    R ca2 = sizeof(R) == 4 ? bn * bn * irho : bn * bn / rho;
    R bt2s = sizeof(R) == 4 ? (bt1 * bt1 + bt2 * bt2) * irho : (bt1 * bt1 + bt2 * bt2) / rho;
    R t = a2 - ca2 - bt2s;
    R disc = t * t + R(4) * a2 * bt2s;
    return Num<R>::sqrt_(R(0.5) * (a2 + ca2 + bt2s + Num<R>::sqrt_(disc)));
}

// ---- seven-wave eigensystem of the 1-D primitive system -----------------
// Roe-Balsara normalisation; waves v-cf, v-ca, v-cs, v, v+cs, v+ca, v+cf.
template <class R> struct Eig {
    R rho, irho, sr, isr, a2, ia2, a, cf, cs, ca, af, as, by, bz, s, vn, nrm;
};

// a2 = gamma P / rho (primitive sound speed squared, Roe-averaged for Roe);
// rsr = 1/sqrt(rho)
template <class R>
__device__ __forceinline__ void eig_setup_r(R rho, R rsr, R vn, R a2, R bn, R bt1, R bt2, Eig<R>& e)
{
    e.rho = rho;
    e.vn = vn;
    R cf2, cs2;
    if constexpr (sizeof(R) == 4) {
        // FP32: square roots and reciprocals from three reciprocal square
        // roots: 1/sqrt(rho) gives sqrt(rho), 1/rho and c_a = |B_n|/sqrt(rho);
        // 1/c_f and 1/a give c_f, a, 1/a^2 and c_s = a c_a / c_f
        // (c_s^2 c_f^2 = a^2 c_a^2)
        e.isr = rsr;
        e.irho = rsr * rsr;
        e.sr = rho * rsr;
        R ca2 = bn * bn * e.irho;
        R bt2s = (bt1 * bt1 + bt2 * bt2) * e.irho;
        R t = a2 - ca2 - bt2s;
        R disc = t * t + R(4) * a2 * bt2s;
        cf2 = R(0.5) * (a2 + ca2 + bt2s + Num<R>::sqrt_(disc));
        const R rcf = Num<R>::rsqrt_(cf2), ra = Num<R>::rsqrt_(a2);
        e.cf = cf2 * rcf;
        e.a = a2 * ra;
        e.ia2 = ra * ra;
        e.ca = Num<R>::abs_(bn) * rsr;
        e.cs = e.a * e.ca * rcf;
        cs2 = e.cs * e.cs;
    } else {
        // FP64: the oracle's chain of correctly rounded divisions and square
        // roots.  Near c_f = c_s the amplitudes below hang on the difference
        // c_f^2 - c_s^2; the few extra ulps of the reciprocal-square-root
        // forms grow there past the 1e-12 parity bar.
        e.irho = R(1) / rho;
        e.sr = Num<R>::sqrt_(rho);
        e.isr = e.sr * e.irho;
        R ca2 = bn * bn * e.irho;
        R bt2s = (bt1 * bt1 + bt2 * bt2) * e.irho;
        R t = a2 - ca2 - bt2s;
        R disc = t * t + R(4) * a2 * bt2s;
        cf2 = R(0.5) * (a2 + ca2 + bt2s + Num<R>::sqrt_(disc));
        cs2 = a2 * ca2 / cf2;
        e.cf = Num<R>::sqrt_(cf2);
        e.cs = Num<R>::sqrt_(cs2);
        e.ca = Num<R>::sqrt_(ca2);
        e.a = Num<R>::sqrt_(a2);
        e.ia2 = R(1) / a2;
    }
    e.a2 = a2;
    R dd = cf2 - cs2;
    // the degenerate limits hold where the quantity is zero up to round-off
    // (a state degenerate in exact arithmetic -- B = 0 carried through a Roe
    // flux -- comes out with B_t of 1e-23, and the basis would follow the
    // direction of that noise): c_f = c_s when c_f^2 - c_s^2 <= 1e-12 c_f^2,
    // B_t = 0 when |B_t|^2 <= 1e-24 (rho a^2 + B_n^2)
    if (dd > R(1e-12) * cf2) {
        R idd = R(1) / dd;
        e.af = Num<R>::sqrt_(rmax(R(0), a2 - cs2) * idd);
        e.as = Num<R>::sqrt_(rmax(R(0), cf2 - a2) * idd);
    } else {
        e.af = R(1);
        e.as = R(0);
    }
    R btm2 = bt1 * bt1 + bt2 * bt2;
    if (btm2 > R(1e-24) * (rho * a2 + bn * bn)) {
        R ibt = sizeof(R) == 4 ? Num<R>::rsqrt_(btm2) : R(1) / Num<R>::sqrt_(btm2);
        e.by = bt1 * ibt;
        e.bz = bt2 * ibt;
    } else {
        e.by = Num<R>::sqrt_(R(0.5));
        e.bz = e.by;
    }
    e.s = sgn1(bn);
    e.nrm = R(0.5) * e.ia2;
}

template <class R>
__device__ __forceinline__ void eig_setup(R rho, R vn, R a2, R bn, R bt1, R bt2, Eig<R>& e)
{
    eig_setup_r(rho, sizeof(R) == 4 ? Num<R>::rsqrt_(rho) : R(0), vn, a2, bn, bt1, bt2, e);
}

// the eigensystem of a cell state from its pressure: a^2 = gamma P / rho with
// the 1/rho of the reciprocal square root
template <class R>
__device__ __forceinline__ void eig_setup_p(R rho, R vn, R gam, R P, R bn, R bt1, R bt2, Eig<R>& e)
{
    if constexpr (sizeof(R) == 4) {
        const R rsr = Num<R>::rsqrt_(rho);
        eig_setup_r(rho, rsr, vn, gam * P * (rsr * rsr), bn, bt1, bt2, e);
    } else {
        eig_setup_r(rho, R(0), vn, gam * P / rho, bn, bt1, bt2, e);   // FP64: the oracle's a^2
    }
}

template <class R>
__device__ __forceinline__ void eig_lambda(const Eig<R>& e, R lam[7])
{
    lam[0] = e.vn - e.cf; lam[1] = e.vn - e.ca; lam[2] = e.vn - e.cs; lam[3] = e.vn;
    lam[4] = e.vn + e.cs; lam[5] = e.vn + e.ca; lam[6] = e.vn + e.cf;
}

// wave amplitudes a = L dw, using the sparsity of the left eigenvectors
template <class R>
__device__ __forceinline__ void eig_project(const Eig<R>& e, const R dw[7], R da[7])
{
    R q = e.by * dw[2] + e.bz * dw[3];              // transverse velocity along beta
    R qb = (e.by * dw[5] + e.bz * dw[6]) * e.isr;   // transverse field along beta
    R av = -e.bz * dw[2] + e.by * dw[3];            // rotational velocity
    R ab = (e.bz * dw[5] - e.by * dw[6]) * e.isr;   // rotational field
    R pr = dw[4] * e.irho;
    R Cf = e.af * e.cf, Cs = e.as * e.cs;
    R fq = e.as * e.cs * e.s, sq = e.af * e.cf * e.s;
    da[0] = e.nrm * (-Cf * dw[1] + fq * q + e.af * pr + e.as * e.a * qb);
    da[6] = e.nrm * ( Cf * dw[1] - fq * q + e.af * pr + e.as * e.a * qb);
    da[2] = e.nrm * (-Cs * dw[1] - sq * q + e.as * pr - e.af * e.a * qb);
    da[4] = e.nrm * ( Cs * dw[1] + sq * q + e.as * pr - e.af * e.a * qb);
    da[1] = R(0.5) * (av - e.s * ab);
    da[5] = R(0.5) * (av + e.s * ab);
    da[3] = dw[0] - dw[4] * e.ia2;
}

// dw = R a, using the sparsity of the right eigenvectors
template <class R>
__device__ __forceinline__ void eig_expand(const Eig<R>& e, const R da[7], R dw[7])
{
    R fs = da[0] + da[6], fd = da[6] - da[0];
    R ss = da[2] + da[4], sd = da[4] - da[2];
    R as_ = da[1] + da[5], ad = da[5] - da[1];
    R tr = e.as * e.cs * (-fd) + e.af * e.cf * sd;   // common transverse-velocity factor
    R bf = e.a * e.sr * (e.as * fs - e.af * ss);       // common transverse-field factor
    dw[0] = e.rho * (e.af * fs + e.as * ss) + da[3];
    dw[1] = e.af * e.cf * fd + e.as * e.cs * sd;
    dw[2] = e.s * e.by * tr - e.bz * as_;
    dw[3] = e.s * e.bz * tr + e.by * as_;
    dw[4] = e.rho * e.a2 * (e.af * fs + e.as * ss);
    dw[5] = e.by * bf + e.s * e.sr * e.bz * ad;
    dw[6] = e.bz * bf - e.s * e.sr * e.by * ad;
}

// P += c r_K: column K of the right eigenvectors (eig_expand of the unit
// amplitude e_K), with its zero entries left out
template <int K, class R>
__device__ __forceinline__ void eig_add_col(const Eig<R>& e, R c, R P[7])
{
    if (K == 3) {                              // entropy wave
        P[0] += c;
        return;
    }
    if (K == 1 || K == 5) {                    // Alfven waves
        const R t = (K == 1 ? R(-1) : R(1)) * e.s * e.sr * c;
        P[2] -= c * e.bz;
        P[3] += c * e.by;
        P[5] += t * e.bz;
        P[6] -= t * e.by;
        return;
    }
    // magnetosonic waves: K = 0, 6 fast, K = 2, 4 slow; sg = -1 on the left-going one
    const bool fast = K == 0 || K == 6;
    const R sg = (K == 0 || K == 2) ? R(-1) : R(1);
    const R A = fast ? e.af : e.as;
    const R Cn = fast ? e.af * e.cf : e.as * e.cs;
    const R tr = fast ? -sg * e.as * e.cs : sg * e.af * e.cf;
    const R bf = fast ? e.a * e.sr * e.as : -(e.a * e.sr * e.af);
    P[0] += c * (e.rho * A);
    P[1] += c * (sg * Cn);
    P[2] += c * (e.s * e.by * tr);
    P[3] += c * (e.s * e.bz * tr);
    P[4] += c * (e.rho * e.a2 * A);
    P[5] += c * (e.by * bf);
    P[6] += c * (e.bz * bf);
}

// ---- Riemann solvers ------------------------------------------------------
template <class R>
__device__ __forceinline__ void hlle_core(const R wl[7], const R wr[7], R bn, R gm1, R gam,
                                          bool have_roe, R roe_vn, R roe_cf, R f[7])
{
    R fl[7], fr[7], ul[7], ur[7];
    phys_flux(wl, bn, gm1, fl);
    phys_flux(wr, bn, gm1, fr);
    to_cons(wl, bn, gm1, ul);
    to_cons(wr, bn, gm1, ur);
    const R irl = R(1) / wl[0], irr = R(1) / wr[0];
    const R a2l = sizeof(R) == 4 ? gam * wl[4] * irl : gam * wl[4] / wl[0];
    const R a2r = sizeof(R) == 4 ? gam * wr[4] * irr : gam * wr[4] / wr[0];
    R cfl = fast_speed(wl[0], irl, a2l, bn, wl[5], wl[6]);
    R cfr = fast_speed(wr[0], irr, a2r, bn, wr[5], wr[6]);
    R sL = wl[1] - cfl, sR = wr[1] + cfr;
    if (have_roe) {
        sL = rmin(sL, roe_vn - roe_cf);
        sR = rmax(sR, roe_vn + roe_cf);
    }
    R bm = rmin(sL, R(0)), bp = rmax(sR, R(0));
    if (bp - bm == R(0)) {
#pragma unroll
        for (int k = 0; k < 7; k++) f[k] = R(0.5) * (fl[k] + fr[k]);
        return;
    }
    R idb = R(1) / (bp - bm);
#pragma unroll
    for (int k = 0; k < 7; k++) f[k] = (bp * fl[k] - bm * fr[k] + bp * bm * (ur[k] - ul[k])) * idb;
}

// Roe averages of the linearisation used by the Roe and HLLE solvers
template <class R> struct RoeAvg {
    R rho, irho, u, v, w, b1, b2, X, a2;
};

template <class R>
__device__ __forceinline__ void roe_average(const R wl[7], const R wr[7], R bn, R gm1, R gam, RoeAvg<R>& m)
{
    // FP32: sqrt(rho) and 1/sqrt(rho) of each side from one reciprocal square
    // root; sqrt(rho) h = (E + p_T) / sqrt(rho) and 1/(sqrt(rho_L) sqrt(rho_R))
    // = 1/rho_Roe without a division.  FP64: the oracle's divisions and
    // square roots (the parity bar; see eig_setup_r)
    constexpr bool F32 = sizeof(R) == 4;
    const R rsl = F32 ? Num<R>::rsqrt_(wl[0]) : R(0), rsr = F32 ? Num<R>::rsqrt_(wr[0]) : R(0);
    R sl = F32 ? wl[0] * rsl : Num<R>::sqrt_(wl[0]), sr = F32 ? wr[0] * rsr : Num<R>::sqrt_(wr[0]);
    R isum = R(1) / (sl + sr);
    m.rho = sl * sr;
    m.irho = F32 ? rsl * rsr : R(1) / m.rho;
    m.u = (sl * wl[1] + sr * wr[1]) * isum;
    m.v = (sl * wl[2] + sr * wr[2]) * isum;
    m.w = (sl * wl[3] + sr * wr[3]) * isum;
    R el = total_energy(wl, bn, gm1), er = total_energy(wr, bn, gm1);
    R h;
    if constexpr (F32) {
        R shl = (el + wl[4] + R(0.5) * (bn * bn + wl[5] * wl[5] + wl[6] * wl[6])) * rsl;   // sqrt(rho_L) h_L
        R shr = (er + wr[4] + R(0.5) * (bn * bn + wr[5] * wr[5] + wr[6] * wr[6])) * rsr;   // sqrt(rho_R) h_R
        h = (shl + shr) * isum;
    } else {
        R hl = (el + wl[4] + R(0.5) * (bn * bn + wl[5] * wl[5] + wl[6] * wl[6])) / wl[0];
        R hr = (er + wr[4] + R(0.5) * (bn * bn + wr[5] * wr[5] + wr[6] * wr[6])) / wr[0];
        h = (sl * hl + sr * hr) * isum;
    }
    m.b1 = (sr * wl[5] + sl * wr[5]) * isum;
    m.b2 = (sr * wl[6] + sl * wr[6]) * isum;
    R d5 = wl[5] - wr[5], d6 = wl[6] - wr[6];
    m.X = R(0.5) * (d5 * d5 + d6 * d6) * isum * isum;
    const R mag = F32 ? (bn * bn + m.b1 * m.b1 + m.b2 * m.b2) * m.irho : (bn * bn + m.b1 * m.b1 + m.b2 * m.b2) / m.rho;
    m.a2 = gm1 * (h - R(0.5) * (m.u * m.u + m.v * m.v + m.w * m.w) - mag) - (gam - R(2)) * m.X;
}

template <class R>
__device__ __forceinline__ void hlle_flux(const R wl[7], const R wr[7], R bn, R gm1, R gam, R f[7])
{
    RoeAvg<R> m;
    roe_average(wl, wr, bn, gm1, gam, m);
    bool ok = m.a2 > R(0);
    R cf = ok ? fast_speed(m.rho, m.irho, m.a2, bn, m.b1, m.b2) : R(0);
    hlle_core(wl, wr, bn, gm1, gam, ok, m.u, cf, f);
}

// conserved image M q of a primitive-space vector q under the Roe state
// (the X term of the linearisation enters through q4 - X q0); the full
// vector, or only the density, momentum, energy and B_t parts used by the
// intermediate-state check (the same thing: all seven)
template <class R>
__device__ __forceinline__ void roe_to_cons(const RoeAvg<R>& m, R ke, R igm1, const R q[7], R u[7])
{
    u[0] = q[0];
    u[1] = m.u * q[0] + m.rho * q[1];
    u[2] = m.v * q[0] + m.rho * q[2];
    u[3] = m.w * q[0] + m.rho * q[3];
    u[4] = (q[4] - m.X * q[0]) * igm1 + ke * q[0] + m.rho * (m.u * q[1] + m.v * q[2] + m.w * q[3])
           + m.b1 * q[5] + m.b2 * q[6];
    u[5] = q[5];
    u[6] = q[6];
}

// intermediate state U_L + M P of the Roe fan: false when rho <= 0 or P <= 0
template <class R>
__device__ __forceinline__ bool roe_state_ok(const RoeAvg<R>& m, R ke, R igm1, const R ul[7], const R P[7], R bn,
                                             R gm1)
{
    R d[7];
    roe_to_cons(m, ke, igm1, P, d);
    R rho = ul[0] + d[0];
    R m1 = ul[1] + d[1], m2 = ul[2] + d[2], m3 = ul[3] + d[3];
    R en = ul[4] + d[4], b1 = ul[5] + d[5], b2 = ul[6] + d[6];
    R p = gm1 * (en - R(0.5) * (m1 * m1 + m2 * m2 + m3 * m3) / rho - R(0.5) * (bn * bn + b1 * b1 + b2 * b2));
    return rho > R(0) && p > R(0);
}

// Roe flux with the exact linearisation; returns true when it fell back to HLLE.
// F = F_L + M R (min(lambda, 0) eta): one eigenvector expansion of the
// left-going waves' strengths; the intermediate states U_L + M sum_{b<=a}
// eta_b r_b are accumulated wave by wave in primitive space.
template <class R>
__device__ __forceinline__ bool roe_flux(const R wl[7], const R wr[7], R bn, R gm1, R gam, R f[7])
{
    RoeAvg<R> m;
    roe_average(wl, wr, bn, gm1, gam, m);
    if (!(m.a2 > R(0))) {
        hlle_core(wl, wr, bn, gm1, gam, false, R(0), R(0), f);
        return true;
    }
    Eig<R> e;
    eig_setup(m.rho, m.u, m.a2, bn, m.b1, m.b2, e);
    R lam[7];
    eig_lambda(e, lam);
    R dq[7];
    dq[0] = wr[0] - wl[0];
    dq[1] = wr[1] - wl[1];
    dq[2] = wr[2] - wl[2];
    dq[3] = wr[3] - wl[3];
    dq[4] = (wr[4] - wl[4]) + m.X * dq[0];
    dq[5] = wr[5] - wl[5];
    dq[6] = wr[6] - wl[6];
    R eta[7];
    eig_project(e, dq, eta);
    const R igm1 = R(1) / gm1;
    const R ke = R(0.5) * (m.u * m.u + m.v * m.v + m.w * m.w) + m.X;
    R ul[7];
    to_cons(wl, bn, gm1, ul);
    // A componentwise bound of the six partial sums P_a = sum_{b<=a} eta_b q_b
    // (primitive space), pushed through |M|, bounds every intermediate state
    // U_a = U_L + M P_a inside a box around U_L; when the lowest pressure over
    // that box is positive (with a margin far above rounding), every state
    // passes the check below, which is then skipped: same decisions, fewer
    // operations on smooth faces.
    bool safe = false;
    {
        const R F = Num<R>::abs_(eta[0]), S = Num<R>::abs_(eta[2]) + Num<R>::abs_(eta[4]);
        const R A = Num<R>::abs_(eta[1]) + Num<R>::abs_(eta[5]), E3 = Num<R>::abs_(eta[3]);
        const R aby = Num<R>::abs_(e.by), abz = Num<R>::abs_(e.bz);
        const R wr_ = e.af * F + e.as * S;                        // density / pressure weight
        const R wt = e.as * e.cs * F + e.af * e.cf * S;           // transverse velocity weight
        const R wb = e.a * e.sr * (e.as * F + e.af * S);          // transverse field weight
        const R Q0 = e.rho * wr_ + E3, Q1 = e.af * e.cf * F + e.as * e.cs * S;
        const R Q2 = aby * wt + abz * A, Q3 = abz * wt + aby * A;
        const R Q4 = e.rho * e.a2 * wr_;
        const R Q5 = aby * wb + e.sr * abz * A, Q6 = abz * wb + e.sr * aby * A;
        const R au = Num<R>::abs_(m.u), av = Num<R>::abs_(m.v), aw = Num<R>::abs_(m.w);
        const R dm1 = au * Q0 + m.rho * Q1, dm2 = av * Q0 + m.rho * Q2, dm3 = aw * Q0 + m.rho * Q3;
        const R dE = (Q4 + m.X * Q0) * igm1 + ke * Q0 + m.rho * (au * Q1 + av * Q2 + aw * Q3) +
                     Num<R>::abs_(m.b1) * Q5 + Num<R>::abs_(m.b2) * Q6;
        const R rmin = ul[0] - Q0;
        if (rmin > Num<R>::fan_margin * ul[0]) {
            const R m1 = Num<R>::abs_(ul[1]) + dm1, m2 = Num<R>::abs_(ul[2]) + dm2, m3 = Num<R>::abs_(ul[3]) + dm3;
            const R b5 = Num<R>::abs_(ul[5]) + Q5, b6 = Num<R>::abs_(ul[6]) + Q6;
            const R lb = (ul[4] - dE) - R(0.5) * (m1 * m1 + m2 * m2 + m3 * m3) / rmin
                         - R(0.5) * (bn * bn + b5 * b5 + b6 * b6);
            safe = lb > Num<R>::fan_margin * (ul[4] + dE);
        }
    }
    R P[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    bool ok = true;
    if (!safe) {
    eig_add_col<0>(e, eta[0], P); ok &= roe_state_ok(m, ke, igm1, ul, P, bn, gm1);
    eig_add_col<1>(e, eta[1], P); ok &= roe_state_ok(m, ke, igm1, ul, P, bn, gm1);
    eig_add_col<2>(e, eta[2], P); ok &= roe_state_ok(m, ke, igm1, ul, P, bn, gm1);
    eig_add_col<3>(e, eta[3], P); ok &= roe_state_ok(m, ke, igm1, ul, P, bn, gm1);
    eig_add_col<4>(e, eta[4], P); ok &= roe_state_ok(m, ke, igm1, ul, P, bn, gm1);
    eig_add_col<5>(e, eta[5], P); ok &= roe_state_ok(m, ke, igm1, ul, P, bn, gm1);
    }
    if (!ok) {
        R cf = fast_speed(m.rho, m.irho, m.a2, bn, m.b1, m.b2);
        hlle_core(wl, wr, bn, gm1, gam, true, m.u, cf, f);
        return true;
    }
    // F = (F_L + F_R)/2 - (1/2) M R (|lambda| eta) equals F_L + M R (min(lambda, 0) eta)
    // exactly, since the exact linearisation gives F_R - F_L = M R (lambda eta):
    // one physical flux instead of two
    R ae[7], D[7], dis[7];
#pragma unroll
    for (int a = 0; a < 7; a++) ae[a] = rmin(lam[a], R(0)) * eta[a];
    eig_expand(e, ae, D);
    roe_to_cons(m, ke, igm1, D, dis);
    R fl[7];
    phys_flux(wl, bn, gm1, fl);
#pragma unroll
    for (int k = 0; k < 7; k++) f[k] = fl[k] + dis[k];
    return false;
}

// HLLD single-star state on one side (Miyoshi & Kusano 2005)
template <class R>
__device__ __forceinline__ void hlld_star(const R w[7], R bn, R gm1, R S, R SM, R pts, R us[7])
{
    R d = w[0] * (S - w[1]);
    R scale = d * (S - SM);
    R den = scale - bn * bn;
    R rs = d / (S - SM);
    R vt1 = w[2], vt2 = w[3], bt1 = w[5], bt2 = w[6];
    if (Num<R>::abs_(den) > Num<R>::hlld_degen * Num<R>::abs_(scale)) {
        R tmp = (SM - w[1]) / den;
        R fac = (d * (S - w[1]) - bn * bn) / den;
        vt1 = w[2] - bn * w[5] * tmp;
        vt2 = w[3] - bn * w[6] * tmp;
        bt1 = w[5] * fac;
        bt2 = w[6] * fac;
    }
    R e = total_energy(w, bn, gm1);
    R pt = w[4] + R(0.5) * (bn * bn + w[5] * w[5] + w[6] * w[6]);
    R vb = w[1] * bn + w[2] * w[5] + w[3] * w[6];
    R vbs = SM * bn + vt1 * bt1 + vt2 * bt2;
    us[0] = rs;
    us[1] = rs * SM;
    us[2] = rs * vt1;
    us[3] = rs * vt2;
    us[4] = ((S - w[1]) * e - pt * w[1] + pts * SM + bn * (vb - vbs)) / (S - SM);
    us[5] = bt1;
    us[6] = bt2;
}

template <class R>
__device__ __forceinline__ void hlld_flux(const R wl[7], const R wr[7], R bn, R gm1, R gam, R f[7])
{
    R fl[7], fr[7];
    phys_flux(wl, bn, gm1, fl);
    phys_flux(wr, bn, gm1, fr);
    const R irl = R(1) / wl[0], irr = R(1) / wr[0];
    const R a2l = sizeof(R) == 4 ? gam * wl[4] * irl : gam * wl[4] / wl[0];
    const R a2r = sizeof(R) == 4 ? gam * wr[4] * irr : gam * wr[4] / wr[0];
    R cfl = fast_speed(wl[0], irl, a2l, bn, wl[5], wl[6]);
    R cfr = fast_speed(wr[0], irr, a2r, bn, wr[5], wr[6]);
    R cmax = rmax(cfl, cfr);
    R SL = rmin(wl[1], wr[1]) - cmax;
    R SR = rmax(wl[1], wr[1]) + cmax;
    if (SL >= R(0)) {
#pragma unroll
        for (int k = 0; k < 7; k++) f[k] = fl[k];
        return;
    }
    if (SR <= R(0)) {
#pragma unroll
        for (int k = 0; k < 7; k++) f[k] = fr[k];
        return;
    }
    R ptl = wl[4] + R(0.5) * (bn * bn + wl[5] * wl[5] + wl[6] * wl[6]);
    R ptr = wr[4] + R(0.5) * (bn * bn + wr[5] * wr[5] + wr[6] * wr[6]);
    R dl = wl[0] * (SL - wl[1]);
    R dr = wr[0] * (SR - wr[1]);
    R idd = R(1) / (dr - dl);
    R SM = (dr * wr[1] - dl * wl[1] - ptr + ptl) * idd;
    R pts = (dr * ptl - dl * ptr + dl * dr * (wr[1] - wl[1])) * idd;
    R usl[7], usr[7];
    hlld_star(wl, bn, gm1, SL, SM, pts, usl);
    hlld_star(wr, bn, gm1, SR, SM, pts, usr);
    R sql = Num<R>::sqrt_(usl[0]), sqr = Num<R>::sqrt_(usr[0]);
    R SsL = SM - Num<R>::abs_(bn) / sql;
    R SsR = SM + Num<R>::abs_(bn) / sqr;
    const bool left = SM >= R(0);
    // the outer side whose fan we are in, selected element by element (a
    // pointer to either array would put both in local memory)
    R wo[7], fo[7], uso[7];
#pragma unroll
    for (int k = 0; k < 7; k++) {
        wo[k] = left ? wl[k] : wr[k];
        fo[k] = left ? fl[k] : fr[k];
        uso[k] = left ? usl[k] : usr[k];
    }
    R So = left ? SL : SR;
    R uo[7];
    to_cons(wo, bn, gm1, uo);
    if ((left && SsL >= R(0)) || (!left && SsR <= R(0))) {
#pragma unroll
        for (int k = 0; k < 7; k++) f[k] = fo[k] + So * (uso[k] - uo[k]);
        return;
    }
    R s = sgn1(bn);
    R inv = R(1) / (sql + sqr);
    R vl1 = usl[2] / usl[0], vl2 = usl[3] / usl[0], vr1 = usr[2] / usr[0], vr2 = usr[3] / usr[0];
    R v1 = (sql * vl1 + sqr * vr1 + (usr[5] - usl[5]) * s) * inv;
    R v2 = (sql * vl2 + sqr * vr2 + (usr[6] - usl[6]) * s) * inv;
    R b1 = (sql * usr[5] + sqr * usl[5] + sql * sqr * (vr1 - vl1) * s) * inv;
    R b2 = (sql * usr[6] + sqr * usl[6] + sql * sqr * (vr2 - vl2) * s) * inv;
    R vbss = SM * bn + v1 * b1 + v2 * b2;
    R rso = uso[0];
    R vo1 = left ? vl1 : vr1, vo2 = left ? vl2 : vr2;
    R vbs = SM * bn + vo1 * uso[5] + vo2 * uso[6];
    R sqo = left ? sql : sqr;
    R Sso = left ? SsL : SsR;
    R ess = left ? uso[4] - sqo * (vbs - vbss) * s : uso[4] + sqo * (vbs - vbss) * s;
    R uss[7] = {rso, rso * SM, rso * v1, rso * v2, ess, b1, b2};
#pragma unroll
    for (int k = 0; k < 7; k++) f[k] = fo[k] + So * (uso[k] - uo[k]) + Sso * (uss[k] - uso[k]);
}

template <int SOLVER, class R>
__device__ __forceinline__ void riemann(const R wl[7], const R wr[7], R bn, R gm1, R gam, R f[7])
{
    if (SOLVER == ROE) roe_flux(wl, wr, bn, gm1, gam, f);
    else if (SOLVER == HLLD) hlld_flux(wl, wr, bn, gm1, gam, f);
    else hlle_flux(wl, wr, bn, gm1, gam, f);
}

// ---- reconstruction -------------------------------------------------------
template <class R>
__device__ __forceinline__ R mc(R l, R r, R c)
{
    // sign of c on the limited magnitude (c = -0 gives -0 where the sign
    // factor gave +0: the same value)
    if (l * r > R(0))
        return Num<R>::copysign_(rmin(rmin(R(2) * Num<R>::abs_(l), R(2) * Num<R>::abs_(r)), Num<R>::abs_(c)), c);
    return R(0);
}

template <class R>
__device__ __forceinline__ R clamp_between(R x, R a, R b)
{
    R lo = rmin(a, b), hi = rmax(a, b);
    return rmin(rmax(x, lo), hi);
}

// characteristic-MC-limited slope dw of the cell with neighbours m, p
template <class R>
__device__ __forceinline__ void char_slope_e(const Eig<R>& e, const R wm[7], const R w0[7], const R wp[7], R dw[7])
{
    R dl[7], dr[7], al[7], ar[7];
#pragma unroll
    for (int k = 0; k < 7; k++) {
        dl[k] = w0[k] - wm[k];
        dr[k] = wp[k] - w0[k];
    }
    eig_project(e, dl, al);
    eig_project(e, dr, ar);
    // the centred difference (w_{+1} - w_{-1})/2 projects to (al + ar)/2 (L is linear)
    R da[7];
#pragma unroll
    for (int a = 0; a < 7; a++) da[a] = mc(al[a], ar[a], R(0.5) * (al[a] + ar[a]));
    eig_expand(e, da, dw);
}

// the eigensystem of a cell state (w, B_n) for the reconstruction and the
// PPM slopes: one set-up serves both
template <class R>
__device__ __forceinline__ void cell_eig(const R w0[7], R bn, R gam, Eig<R>& e)
{
    eig_setup_p(w0[0], w0[1], gam, w0[4], bn, w0[5], w0[6], e);
}

template <class R>
__device__ __forceinline__ void char_slope(const R wm[7], const R w0[7], const R wp[7], R bn, R gam, R dw[7])
{
    Eig<R> e;
    cell_eig(w0, bn, gam, e);
    char_slope_e(e, wm, w0, wp, dw);
}

// Face states of one cell: wm on its face -1/2, wp on its face +1/2.
// w0 the cell, wm1/wp1 its neighbours; for PPM, dwm/dw0/dwp are the
// characteristic-limited slopes of cells -1, 0, +1.  trace: CTU tracing
// with dtdx = dt/dx.
template <int RECON, bool TRACE, class R>
__device__ __forceinline__ void recon_cell_e(const Eig<R>& e, const R wm1[7], const R w0[7], const R wp1[7],
                                             const R dwm[7], const R dw0[7], const R dwp[7], R dtdx,
                                             R wm[7], R wp[7])
{
    R pl[7], pr[7];
    if (RECON == PLM) {
        R dl[7], dr[7], al[7], ar[7];
#pragma unroll
        for (int k = 0; k < 7; k++) {
            dl[k] = w0[k] - wm1[k];
            dr[k] = wp1[k] - w0[k];
        }
        eig_project(e, dl, al);
        eig_project(e, dr, ar);
#pragma unroll
        for (int a = 0; a < 7; a++) {
            R d = mc(al[a], ar[a], R(0.5) * (al[a] + ar[a]));
            pl[a] = R(-0.5) * d;
            pr[a] = R(0.5) * d;
        }
    } else {
        R fm[7], fp[7];
#pragma unroll
        for (int k = 0; k < 7; k++) {
            R vm = R(0.5) * (wm1[k] + w0[k]) - (dw0[k] - dwm[k]) * R(1.0 / 6.0);
            R vp = R(0.5) * (w0[k] + wp1[k]) - (dwp[k] - dw0[k]) * R(1.0 / 6.0);
            fm[k] = clamp_between(vm, wm1[k], w0[k]) - w0[k];
            fp[k] = clamp_between(vp, w0[k], wp1[k]) - w0[k];
        }
        eig_project(e, fm, pl);
        eig_project(e, fp, pr);
#pragma unroll
        for (int a = 0; a < 7; a++) {
            R l = pl[a], r = pr[a];
            if (l * r >= R(0)) {
                l = R(0);
                r = R(0);
            } else {
                R dlt = r - l, a6 = R(-3) * (l + r);
                if (dlt * a6 > dlt * dlt) l = R(-2) * r;
                else if (-dlt * dlt > dlt * a6) r = R(-2) * l;
            }
            pl[a] = l;
            pr[a] = r;
        }
    }
    if (TRACE) {
        R lam[7];
        eig_lambda(e, lam);
        R smax = rmax(lam[6], R(0)) * dtdx;
        R smin = rmin(lam[0], R(0)) * dtdx;
#pragma unroll
        for (int a = 0; a < 7; a++) {
            R dlt = pr[a] - pl[a], a6 = R(-3) * (pl[a] + pr[a]);
            R sp = lam[a] > R(0) ? lam[a] * dtdx : smax;
            R sm = lam[a] < R(0) ? lam[a] * dtdx : smin;
            R r_ = pr[a] - R(0.5) * sp * (dlt - (R(1) - R(2) / R(3) * sp) * a6);
            R l_ = pl[a] - R(0.5) * sm * (dlt + (R(1) + R(2) / R(3) * sm) * a6);
            pl[a] = l_;
            pr[a] = r_;
        }
    }
    R dm[7], dp[7];
    eig_expand(e, pr, dp);
    if (RECON == PLM && !TRACE) {
        // pl = -pr, and the expansion is odd in its argument
#pragma unroll
        for (int k = 0; k < 7; k++) dm[k] = -dp[k];
    } else {
        eig_expand(e, pl, dm);
    }
#pragma unroll
    for (int k = 0; k < 7; k++) {
        wm[k] = w0[k] + dm[k];
        wp[k] = w0[k] + dp[k];
        if (!TRACE) {
            wm[k] = clamp_between(wm[k], wm1[k], w0[k]);
            wp[k] = clamp_between(wp[k], w0[k], wp1[k]);
        }
    }
}

template <int RECON, bool TRACE, class R>
__device__ __forceinline__ void recon_cell(const R wm1[7], const R w0[7], const R wp1[7], R bn, R gam,
                                           const R dwm[7], const R dw0[7], const R dwp[7], R dtdx,
                                           R wm[7], R wp[7])
{
    if (RECON == PLM_PRIM) {
#pragma unroll
        for (int k = 0; k < 7; k++) {
            R d = mc(w0[k] - wm1[k], wp1[k] - w0[k], R(0.5) * (wp1[k] - wm1[k]));
            wm[k] = w0[k] - R(0.5) * d;
            wp[k] = w0[k] + R(0.5) * d;
        }
        return;
    }
    Eig<R> e;
    cell_eig(w0, bn, gam, e);
    recon_cell_e<RECON, TRACE>(e, wm1, w0, wp1, dwm, dw0, dwp, dtdx, wm, wp);
}

}  // namespace mhd
