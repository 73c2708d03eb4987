/*
 * mhd_oracle.c -- plain, slow FP64 CPU oracle of the ideal-MHD patch advance
 * (unsplit VL and CTU schemes with constrained transport) of
 * "Magnetohydrodynamics with GAMER" (Zhang, Schive & Chiueh 2018).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, import or
 * call this file: only tests/, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header or constant with the CUDA library.
 *
 * Build:  gcc -O2 -std=c99 -ffp-contract=off -fopenmp -shared -fPIC
 * (-ffp-contract=off: every a*b+c is rounded twice, as written.)
 *
 * Storage (periodic box, no duplicated face):
 *   U[f*n + c], f = 0..4 : rho, Mx, My, Mz, e          (cell averages, Eq. 11)
 *   B[d*n + c], d = 0..2 : B_d on the face c - 1/2 e_d  (face averages, Eq. 14)
 *   c = (k*ny + j)*nx + i,  n = nx*ny*nz,  dx = dy = dz (Sec. 3.1).
 *
 * Readings of the paper taken here (the paper defers the scheme details to
 * the ATHENA papers it cites in Sec. 3.2) are listed in the repository's
 * design notes; each function below states the passage it follows.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Stage marks: nothing in this build.  The operation-counting build         */
/* (flopcount.cpp, the same source with a counting scalar type) attributes   */
/* the operations done since the previous mark to the named stage.           */
#ifndef ORC_STAGE
#define ORC_STAGE(name)
#endif

enum { VL = 0, CTU = 1 };
enum { PLM = 0, PPM = 1, PLM_PRIM = 2 };
enum { ROE = 0, HLLD = 1, HLLE = 2 };

typedef struct {
    int nx, ny, nz;
    long n;
    double dx, gam;
    double pfloor;   /* pressure floor, 0 = none (see prim_floor) */
    int bc;          /* bit d set: outflow (zero-gradient) boundaries along axis d, else periodic */
} grid_t;

/* index along an axis of n cells: periodic wrap, or for an outflow axis the */
/* nearest cell (zero-gradient ghost cells; the same rule maps the face or    */
/* edge beyond the last cell onto the last one, so the outer face field and   */
/* edge fields continue the last interior ones)                               */
static int bidx(int i, int n, int outflow)
{
    if (outflow) return i < 0 ? 0 : (i >= n ? n - 1 : i);
    i %= n;
    return i < 0 ? i + n : i;
}

static long cidx(const grid_t *g, int i, int j, int k)
{
    i = bidx(i, g->nx, g->bc & 1);
    j = bidx(j, g->ny, g->bc & 2);
    k = bidx(k, g->nz, g->bc & 4);
    return ((long)k * g->ny + j) * g->nx + i;
}

/* neighbour of cell c shifted by s along axis d (periodic or outflow) */
static long shift(const grid_t *g, long c, int d, int s)
{
    int i = (int)(c % g->nx), j = (int)((c / g->nx) % g->ny), k = (int)(c / ((long)g->nx * g->ny));
    if (d == 0) i += s; else if (d == 1) j += s; else k += s;
    return cidx(g, i, j, k);
}

static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }
static double sgn1(double a) { return a >= 0.0 ? 1.0 : -1.0; }

/* ------------------------------------------------------------------------ */
/* Eq. 5: total energy and its inverse, the gas pressure.                    */
/* 1-D primitive vector in the frame of a sweep along n (t1, t2 cyclic):     */
/*   w = (rho, v_n, v_t1, v_t2, P, B_t1, B_t2), B_n separate.                 */
/* ------------------------------------------------------------------------ */
static double energy_of(const double w[7], double bn, double gam)
{
    double v2 = w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
    double b2 = bn * bn + w[5] * w[5] + w[6] * w[6];
    return w[4] / (gam - 1.0) + 0.5 * w[0] * v2 + 0.5 * b2;
}

/* 1-D conserved vector (rho, M_n, M_t1, M_t2, e, B_t1, B_t2) of w */
static void cons_of(const double w[7], double bn, double gam, double u[7])
{
    u[0] = w[0];
    u[1] = w[0] * w[1];
    u[2] = w[0] * w[2];
    u[3] = w[0] * w[3];
    u[4] = energy_of(w, bn, gam);
    u[5] = w[5];
    u[6] = w[6];
}

/* Eqs. 7-9, the flux along n in the sweep frame (the B_n row is zero) */
void orc_flux_phys(const double w[7], double bn, double gam, double f[7])
{
    double e = energy_of(w, bn, gam);
    double b2 = bn * bn + w[5] * w[5] + w[6] * w[6];
    double pt = w[4] + 0.5 * b2;
    double vb = w[1] * bn + w[2] * w[5] + w[3] * w[6];
    f[0] = w[0] * w[1];
    f[1] = w[0] * w[1] * w[1] + pt - bn * bn;
    f[2] = w[0] * w[1] * w[2] - bn * w[5];
    f[3] = w[0] * w[1] * w[3] - bn * w[6];
    f[4] = (e + pt) * w[1] - bn * vb;
    f[5] = w[5] * w[1] - bn * w[2];
    f[6] = w[6] * w[1] - bn * w[3];
}

/* fast magnetosonic speed along n for sound speed squared a2 */
static double fast_speed(double rho, double a2, double bn, double bt1, double bt2)
{
    double ca2 = bn * bn / rho;
    double bt2s = (bt1 * bt1 + bt2 * bt2) / rho;
    double t = a2 - ca2 - bt2s;
    double disc = t * t + 4.0 * a2 * bt2s;
    return sqrt(0.5 * (a2 + ca2 + bt2s + sqrt(disc)));
}

/* ------------------------------------------------------------------------ */
/* Seven-wave eigensystem of the 1-D primitive MHD system (B_n held fixed),  */
/* the characteristic basis the reconstruction of CTU/VL step 1 (Sec. 3.2)   */
/* projects on.  rho*a2 plays the role of gamma*P.  Waves in order           */
/*   v-cf, v-ca, v-cs, v, v+cs, v+ca, v+cf.                                   */
/* R[k][a]: component k of right eigenvector a.  L[a][k]: left eigenvectors, */
/* normalised so that L R = I.                                                */
/* ------------------------------------------------------------------------ */
#define EIG_DEGEN_CF 1e-12
#define EIG_DEGEN_BT 1e-24
static void eigen7(double rho, double vn, double a2, double bn, double bt1, double bt2,
                   double lam[7], double R[7][7], double L[7][7])
{
    double sr = sqrt(rho);
    double ca2 = bn * bn / rho;
    double bt2s = (bt1 * bt1 + bt2 * bt2) / rho;
    double t = a2 - ca2 - bt2s;
    double disc = t * t + 4.0 * a2 * bt2s;
    double cf2 = 0.5 * (a2 + ca2 + bt2s + sqrt(disc));
    double cs2 = a2 * ca2 / cf2;
    double cf = sqrt(cf2), cs = sqrt(cs2), ca = sqrt(ca2), a = sqrt(a2);
    double dd = cf2 - cs2;
    double af, as;
    /* degenerate limits, taken where the quantity is zero up to round-off   */
    /* (a state that is degenerate in exact arithmetic, e.g. B = 0 carried   */
    /* through a Roe flux, comes out with B_t of 1e-23; the basis would then */
    /* follow the direction of the rounding noise): c_f = c_s when           */
    /* c_f^2 - c_s^2 <= EIG_DEGEN_CF c_f^2, B_t = 0 when                     */
    /* |B_t|^2 <= EIG_DEGEN_BT (rho a^2 + B_n^2)                              */
    if (dd > EIG_DEGEN_CF * cf2) {
        af = sqrt(dmax(0.0, a2 - cs2) / dd);
        as = sqrt(dmax(0.0, cf2 - a2) / dd);
    } else {
        af = 1.0; as = 0.0;
    }
    double btm2 = bt1 * bt1 + bt2 * bt2;
    double by, bz;
    if (btm2 > EIG_DEGEN_BT * (rho * a2 + bn * bn)) {
        double btm = sqrt(btm2);
        by = bt1 / btm; bz = bt2 / btm;
    } else {
        by = sqrt(0.5); bz = sqrt(0.5);
    }
    double s = sgn1(bn);
    double nrm = 0.5 / a2;

    lam[0] = vn - cf; lam[1] = vn - ca; lam[2] = vn - cs; lam[3] = vn;
    lam[4] = vn + cs; lam[5] = vn + ca; lam[6] = vn + cf;

    /* right eigenvectors, columns */
    double col[7][7] = {
        { rho * af, -af * cf,  as * cs * s * by,  as * cs * s * bz, rho * af * a2,  as * a * sr * by,  as * a * sr * bz},
        { 0.0,       0.0,     -bz,                by,               0.0,           -bz * sr * s,       by * sr * s},
        { rho * as, -as * cs, -af * cf * s * by, -af * cf * s * bz, rho * as * a2, -af * a * sr * by, -af * a * sr * bz},
        { 1.0,       0.0,      0.0,               0.0,              0.0,            0.0,               0.0},
        { rho * as,  as * cs,  af * cf * s * by,  af * cf * s * bz, rho * as * a2, -af * a * sr * by, -af * a * sr * bz},
        { 0.0,       0.0,     -bz,                by,               0.0,            bz * sr * s,      -by * sr * s},
        { rho * af,  af * cf, -as * cs * s * by, -as * cs * s * bz, rho * af * a2,  as * a * sr * by,  as * a * sr * bz},
    };
    /* left eigenvectors, rows */
    double row[7][7] = {
        {0.0, -nrm * af * cf,  nrm * as * cs * s * by,  nrm * as * cs * s * bz, nrm * af / rho,  nrm * as * a * by / sr,  nrm * as * a * bz / sr},
        {0.0,  0.0,           -0.5 * bz,                0.5 * by,               0.0,            -0.5 * bz * s / sr,      0.5 * by * s / sr},
        {0.0, -nrm * as * cs, -nrm * af * cf * s * by, -nrm * af * cf * s * bz, nrm * as / rho, -nrm * af * a * by / sr, -nrm * af * a * bz / sr},
        {1.0,  0.0,            0.0,                     0.0,                    -1.0 / a2,       0.0,                     0.0},
        {0.0,  nrm * as * cs,  nrm * af * cf * s * by,  nrm * af * cf * s * bz, nrm * as / rho, -nrm * af * a * by / sr, -nrm * af * a * bz / sr},
        {0.0,  0.0,           -0.5 * bz,                0.5 * by,               0.0,             0.5 * bz * s / sr,     -0.5 * by * s / sr},
        {0.0,  nrm * af * cf, -nrm * as * cs * s * by, -nrm * as * cs * s * bz, nrm * af / rho,  nrm * as * a * by / sr,  nrm * as * a * bz / sr},
    };
    for (int k = 0; k < 7; k++)
        for (int m = 0; m < 7; m++) { R[k][m] = col[m][k]; L[m][k] = row[m][k]; }
}

/* exported for the tests: eigensystem of the cell state w */
void orc_eigen(const double w[7], double bn, double gam, double lam[7], double Rf[49], double Lf[49])
{
    double R[7][7], L[7][7];
    eigen7(w[0], w[1], gam * w[4] / w[0], bn, w[5], w[6], lam, R, L);
    for (int k = 0; k < 7; k++)
        for (int m = 0; m < 7; m++) { Rf[k * 7 + m] = R[k][m]; Lf[k * 7 + m] = L[k][m]; }
}

/* ------------------------------------------------------------------------ */
/* Riemann solvers of CTU step 2 / VL step 1 (Sec. 3.2): HLLE, HLLD, Roe.    */
/* ------------------------------------------------------------------------ */

/* Roe linearisation.  With Roe averages rho~ = sqrt(rhoL rhoR), u~, H~, the  */
/* cross-weighted B~_t = (sqrt(rhoR) B_tL + sqrt(rhoL) B_tR)/(sqrt(rhoL)+     */
/* sqrt(rhoR)) and X = |dB_t|^2 / (2 (sqrt(rhoL)+sqrt(rhoR))^2), the jumps of */
/* U and F are exactly linear in the primitive jumps; in the variables       */
/* (rho, u, v, w, P + X rho, B_t) the matrix is the primitive Jacobian at the */
/* averaged state with sound speed                                           */
/*   a~^2 = (gamma-1)(H~ - |u~|^2/2 - |B~|^2/rho~) - (gamma-2) X.              */
/* Returns 0 if a~^2 <= 0 (no linearisation), else fills the waves.          */
typedef struct {
    double lam[7];
    double eta[7];      /* wave strengths */
    double ru[7][7];    /* ru[a][k]: conserved right eigenvector a */
    double cf;          /* fast speed of the averaged state */
    double vn;
} roe_t;

static int roe_linearise(const double wl[7], const double wr[7], double bn, double gam, roe_t *r)
{
    double sl = sqrt(wl[0]), sr = sqrt(wr[0]);
    double isum = 1.0 / (sl + sr);
    double rho = sl * sr;
    double u = (sl * wl[1] + sr * wr[1]) * isum;
    double v = (sl * wl[2] + sr * wr[2]) * isum;
    double w = (sl * wl[3] + sr * wr[3]) * isum;
    double el = energy_of(wl, bn, gam), er = energy_of(wr, bn, gam);
    double hl = (el + wl[4] + 0.5 * (bn * bn + wl[5] * wl[5] + wl[6] * wl[6])) / wl[0];
    double hr = (er + wr[4] + 0.5 * (bn * bn + wr[5] * wr[5] + wr[6] * wr[6])) / wr[0];
    double h = (sl * hl + sr * hr) * isum;
    double b1 = (sr * wl[5] + sl * wr[5]) * isum;
    double b2 = (sr * wl[6] + sl * wr[6]) * isum;
    double d5 = wl[5] - wr[5], d6 = wl[6] - wr[6];
    double X = 0.5 * (d5 * d5 + d6 * d6) * isum * isum;
    double a2 = (gam - 1.0) * (h - 0.5 * (u * u + v * v + w * w) - (bn * bn + b1 * b1 + b2 * b2) / rho)
                - (gam - 2.0) * X;
    if (!(a2 > 0.0)) return 0;
    double R[7][7], L[7][7];
    eigen7(rho, u, a2, bn, b1, b2, r->lam, R, L);
    r->cf = r->lam[6] - u;
    r->vn = u;
    double dq[7];
    dq[0] = wr[0] - wl[0];
    dq[1] = wr[1] - wl[1];
    dq[2] = wr[2] - wl[2];
    dq[3] = wr[3] - wl[3];
    dq[4] = (wr[4] - wl[4]) + X * dq[0];
    dq[5] = wr[5] - wl[5];
    dq[6] = wr[6] - wl[6];
    for (int a = 0; a < 7; a++) {
        double s = 0.0;
        for (int k = 0; k < 7; k++) s += L[a][k] * dq[k];
        r->eta[a] = s;
        /* right eigenvector back in (rho, u, v, w, P, B_t) then in U */
        double q0 = R[0][a], q1 = R[1][a], q2 = R[2][a], q3 = R[3][a];
        double q4 = R[4][a] - X * R[0][a], q5 = R[5][a], q6 = R[6][a];
        r->ru[a][0] = q0;
        r->ru[a][1] = u * q0 + rho * q1;
        r->ru[a][2] = v * q0 + rho * q2;
        r->ru[a][3] = w * q0 + rho * q3;
        r->ru[a][4] = q4 / (gam - 1.0) + (0.5 * (u * u + v * v + w * w) + X) * q0
                      + rho * (u * q1 + v * q2 + w * q3) + b1 * q5 + b2 * q6;
        r->ru[a][5] = q5;
        r->ru[a][6] = q6;
    }
    return 1;
}

/* exported for the Roe-property test: dF = sum_a lam_a eta_a r_a */
int orc_roe_waves(const double wl[7], const double wr[7], double bn, double gam,
                  double lam[7], double eta[7], double ru[49])
{
    roe_t r;
    if (!roe_linearise(wl, wr, bn, gam, &r)) return 0;
    for (int a = 0; a < 7; a++) {
        lam[a] = r.lam[a];
        eta[a] = r.eta[a];
        for (int k = 0; k < 7; k++) ru[a * 7 + k] = r.ru[a][k];
    }
    return 1;
}

static void hlle_flux(const double wl[7], const double wr[7], double bn, double gam, double f[7])
{
    double fl[7], fr[7], ul[7], ur[7];
    orc_flux_phys(wl, bn, gam, fl);
    orc_flux_phys(wr, bn, gam, fr);
    cons_of(wl, bn, gam, ul);
    cons_of(wr, bn, gam, ur);
    double cfl = fast_speed(wl[0], gam * wl[4] / wl[0], bn, wl[5], wl[6]);
    double cfr = fast_speed(wr[0], gam * wr[4] / wr[0], bn, wr[5], wr[6]);
    double sL = wl[1] - cfl, sR = wr[1] + cfr;
    roe_t r;
    if (roe_linearise(wl, wr, bn, gam, &r)) {   /* Einfeldt speeds */
        sL = dmin(sL, r.vn - r.cf);
        sR = dmax(sR, r.vn + r.cf);
    }
    double bm = dmin(sL, 0.0), bp = dmax(sR, 0.0);
    if (bp - bm == 0.0) {
        for (int k = 0; k < 7; k++) f[k] = 0.5 * (fl[k] + fr[k]);
        return;
    }
    double idb = 1.0 / (bp - bm);
    for (int k = 0; k < 7; k++)
        f[k] = (bp * fl[k] - bm * fr[k] + bp * bm * (ur[k] - ul[k])) * idb;
}

/* Roe flux, no entropy fix; falls back to HLLE when the linearisation does  */
/* not exist or one of its six intermediate states has rho <= 0 or P <= 0.   */
static int roe_flux(const double wl[7], const double wr[7], double bn, double gam, double f[7])
{
    roe_t r;
    double fl[7], fr[7], ul[7];
    if (!roe_linearise(wl, wr, bn, gam, &r)) { hlle_flux(wl, wr, bn, gam, f); return 1; }
    cons_of(wl, bn, gam, ul);
    double us[7];
    for (int k = 0; k < 7; k++) us[k] = ul[k];
    for (int a = 0; a < 6; a++) {
        for (int k = 0; k < 7; k++) us[k] += r.eta[a] * r.ru[a][k];
        double rho = us[0];
        if (!(rho > 0.0)) { hlle_flux(wl, wr, bn, gam, f); return 1; }
        double p = (gam - 1.0) * (us[4] - 0.5 * (us[1] * us[1] + us[2] * us[2] + us[3] * us[3]) / rho
                                  - 0.5 * (bn * bn + us[5] * us[5] + us[6] * us[6]));
        if (!(p > 0.0)) { hlle_flux(wl, wr, bn, gam, f); return 1; }
    }
    orc_flux_phys(wl, bn, gam, fl);
    orc_flux_phys(wr, bn, gam, fr);
    for (int k = 0; k < 7; k++) {
        double d = 0.0;
        for (int a = 0; a < 7; a++) d += fabs(r.lam[a]) * r.eta[a] * r.ru[a][k];
        f[k] = 0.5 * (fl[k] + fr[k]) - 0.5 * d;
    }
    return 0;
}

/* HLLD (Miyoshi & Kusano 2005): five waves S_L, S*_L, S_M, S*_R, S_R.       */
#define HLLD_DEGEN 1e-8
static void hlld_star(const double w[7], double bn, double gam, double S, double SM, double pts,
                      double us[7], double *rhos)
{
    /* single-star state on one side (MK05 Sec. 3) */
    double d = w[0] * (S - w[1]);
    double scale = d * (S - SM);
    double den = scale - bn * bn;
    double rs = d / (S - SM);
    double vt1 = w[2], vt2 = w[3], bt1 = w[5], bt2 = w[6];
    if (fabs(den) > HLLD_DEGEN * fabs(scale)) {
        double tmp = (SM - w[1]) / den;
        double fac = (d * (S - w[1]) - bn * bn) / den;
        vt1 = w[2] - bn * w[5] * tmp;
        vt2 = w[3] - bn * w[6] * tmp;
        bt1 = w[5] * fac;
        bt2 = w[6] * fac;
    }
    double e = energy_of(w, bn, gam);
    double pt = w[4] + 0.5 * (bn * bn + w[5] * w[5] + w[6] * w[6]);
    double vb = w[1] * bn + w[2] * w[5] + w[3] * w[6];
    double vbs = SM * bn + vt1 * bt1 + vt2 * bt2;
    double es = ((S - w[1]) * e - pt * w[1] + pts * SM + bn * (vb - vbs)) / (S - SM);
    us[0] = rs; us[1] = rs * SM; us[2] = rs * vt1; us[3] = rs * vt2;
    us[4] = es; us[5] = bt1; us[6] = bt2;
    *rhos = rs;
}

/* The HLLD fan (MK05): wave speeds S[0..4] = S_L, S*_L, S_M, S*_R, S_R and */
/* the six conserved states U[0..5] = U_L, U*_L, U**_L, U**_R, U*_R, U_R     */
/* between them, with the outer physical fluxes fl, fr.  S_L/S_R =          */
/* min/max(u) -/+ max(c_f); S_M and p_T* from the HLL averages; the single-  */
/* star states from hlld_star; S*_{L,R} = S_M -/+ |B_n|/sqrt(rho*); the      */
/* double-star transverse v and B are the sqrt(rho*)-weighted averages with  */
/* the rotational jump conditions, and each side's e** follows from the     */
/* jump of v.B across its Alfven wave.  When S_L >= 0 or S_R <= 0 the       */
/* interior states are not used (the flux is the upwind one).               */
static void hlld_fan(const double wl[7], const double wr[7], double bn, double gam, double S[5],
                     double U[6][7], double fl[7], double fr[7])
{
    orc_flux_phys(wl, bn, gam, fl);
    orc_flux_phys(wr, bn, gam, fr);
    double cfl = fast_speed(wl[0], gam * wl[4] / wl[0], bn, wl[5], wl[6]);
    double cfr = fast_speed(wr[0], gam * wr[4] / wr[0], bn, wr[5], wr[6]);
    double cmax = dmax(cfl, cfr);
    double SL = dmin(wl[1], wr[1]) - cmax;
    double SR = dmax(wl[1], wr[1]) + cmax;
    double *ul = U[0], *ur = U[5], *usl = U[1], *usr = U[4];
    cons_of(wl, bn, gam, ul);
    cons_of(wr, bn, gam, ur);
    double ptl = wl[4] + 0.5 * (bn * bn + wl[5] * wl[5] + wl[6] * wl[6]);
    double ptr = wr[4] + 0.5 * (bn * bn + wr[5] * wr[5] + wr[6] * wr[6]);
    double dl = wl[0] * (SL - wl[1]);
    double dr = wr[0] * (SR - wr[1]);
    double idd = 1.0 / (dr - dl);
    double SM = (dr * wr[1] - dl * wl[1] - ptr + ptl) * idd;
    double pts = (dr * ptl - dl * ptr + dl * dr * (wr[1] - wl[1])) * idd;
    double rsl, rsr;
    hlld_star(wl, bn, gam, SL, SM, pts, usl, &rsl);
    hlld_star(wr, bn, gam, SR, SM, pts, usr, &rsr);
    double sql = sqrt(rsl), sqr = sqrt(rsr);
    double SsL = SM - fabs(bn) / sql;
    double SsR = SM + fabs(bn) / sqr;
    /* double-star states (rotational discontinuities) */
    double s = sgn1(bn);
    double inv = 1.0 / (sql + sqr);
    double vl1 = usl[2] / rsl, vl2 = usl[3] / rsl, vr1 = usr[2] / rsr, vr2 = usr[3] / rsr;
    double v1 = (sql * vl1 + sqr * vr1 + (usr[5] - usl[5]) * s) * inv;
    double v2 = (sql * vl2 + sqr * vr2 + (usr[6] - usl[6]) * s) * inv;
    double b1 = (sql * usr[5] + sqr * usl[5] + sql * sqr * (vr1 - vl1) * s) * inv;
    double b2 = (sql * usr[6] + sqr * usl[6] + sql * sqr * (vr2 - vl2) * s) * inv;
    double vbss = SM * bn + v1 * b1 + v2 * b2;
    double vbsl = SM * bn + vl1 * usl[5] + vl2 * usl[6];
    double vbsr = SM * bn + vr1 * usr[5] + vr2 * usr[6];
    double ussl[7] = {rsl, rsl * SM, rsl * v1, rsl * v2, usl[4] - sql * (vbsl - vbss) * s, b1, b2};
    double ussr[7] = {rsr, rsr * SM, rsr * v1, rsr * v2, usr[4] + sqr * (vbsr - vbss) * s, b1, b2};
    for (int k = 0; k < 7; k++) { U[2][k] = ussl[k]; U[3][k] = ussr[k]; }
    S[0] = SL; S[1] = SsL; S[2] = SM; S[3] = SsR; S[4] = SR;
}

/* HLLD flux: the upwind flux plus the jumps across the waves on the side  */
/* of x/t = 0 it is taken from (Rankine-Hugoniot across each wave).         */
static void hlld_flux(const double wl[7], const double wr[7], double bn, double gam, double f[7])
{
    double fl[7], fr[7], S[5], U[6][7];
    hlld_fan(wl, wr, bn, gam, S, U, fl, fr);
    if (S[0] >= 0.0) { for (int k = 0; k < 7; k++) f[k] = fl[k]; return; }
    if (S[4] <= 0.0) { for (int k = 0; k < 7; k++) f[k] = fr[k]; return; }
    if (S[1] >= 0.0) {
        for (int k = 0; k < 7; k++) f[k] = fl[k] + S[0] * (U[1][k] - U[0][k]);
        return;
    }
    if (S[3] <= 0.0) {
        for (int k = 0; k < 7; k++) f[k] = fr[k] + S[4] * (U[4][k] - U[5][k]);
        return;
    }
    if (S[2] >= 0.0) {
        for (int k = 0; k < 7; k++) f[k] = fl[k] + S[0] * (U[1][k] - U[0][k]) + S[1] * (U[2][k] - U[1][k]);
    } else {
        for (int k = 0; k < 7; k++) f[k] = fr[k] + S[4] * (U[4][k] - U[5][k]) + S[3] * (U[3][k] - U[4][k]);
    }
}

/* exported: the HLLD fan (speeds S[5], states U[6][7] as in hlld_fan)      */
void orc_hlld_fan(const double wl[7], const double wr[7], double bn, double gam, double S[5], double U[42])
{
    double fl[7], fr[7];
    hlld_fan(wl, wr, bn, gam, S, (double (*)[7])U, fl, fr);
}

/* exported: the HLLE fan, Einfeldt speeds S[0] = S_L, S[1] = S_R (before   */
/* the clamp at 0 the flux applies) and the HLL average state between them */
/* U_hll = (S_R U_R - S_L U_L - (F_R - F_L)) / (S_R - S_L)                   */
void orc_hlle_fan(const double wl[7], const double wr[7], double bn, double gam, double S[2], double Uhll[7])
{
    double fl[7], fr[7], ul[7], ur[7];
    orc_flux_phys(wl, bn, gam, fl);
    orc_flux_phys(wr, bn, gam, fr);
    cons_of(wl, bn, gam, ul);
    cons_of(wr, bn, gam, ur);
    double cfl = fast_speed(wl[0], gam * wl[4] / wl[0], bn, wl[5], wl[6]);
    double cfr = fast_speed(wr[0], gam * wr[4] / wr[0], bn, wr[5], wr[6]);
    double sL = wl[1] - cfl, sR = wr[1] + cfr;
    roe_t r;
    if (roe_linearise(wl, wr, bn, gam, &r)) {
        sL = dmin(sL, r.vn - r.cf);
        sR = dmax(sR, r.vn + r.cf);
    }
    S[0] = sL; S[1] = sR;
    for (int k = 0; k < 7; k++) Uhll[k] = (sR * ur[k] - sL * ul[k] - (fr[k] - fl[k])) / (sR - sL);
}

/* exported: solver 0 Roe, 1 HLLD, 2 HLLE; returns 1 if Roe fell back to HLLE */
int orc_riemann(int solver, const double wl[7], const double wr[7], double bn, double gam, double f[7])
{
    if (solver == ROE) return roe_flux(wl, wr, bn, gam, f);
    if (solver == HLLD) { hlld_flux(wl, wr, bn, gam, f); return 0; }
    hlle_flux(wl, wr, bn, gam, f);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 1-D reconstruction of CTU step 1 / VL step 4 (Sec. 3.2).                  */
/* Input: primitive states of cells i-2..i+2 along the sweep (w5[m], m=0..4, */
/* the cell itself at m=2), the cell-centred B_n of each, the time step over */
/* dx (used only when trace != 0).  Output: the state on the face i-1/2      */
/* (wm) and on the face i+1/2 (wp), both as seen from cell i.                */
/* ------------------------------------------------------------------------ */
static double mc_limit(double dl, double dr, double dc)
{
    if (dl * dr > 0.0)
        return sgn1(dc) * dmin(dmin(2.0 * fabs(dl), 2.0 * fabs(dr)), fabs(dc));
    return 0.0;
}

/* characteristic-limited slope dW of cell m (MC limiter per wave) */
static void char_slope(const double wm1[7], const double w0[7], const double wp1[7], double bn, double gam,
                       double dw[7])
{
    double lam[7], R[7][7], L[7][7];
    eigen7(w0[0], w0[1], gam * w0[4] / w0[0], bn, w0[5], w0[6], lam, R, L);
    double da[7];
    for (int a = 0; a < 7; a++) {
        double al = 0.0, ar = 0.0, ac = 0.0;
        for (int k = 0; k < 7; k++) {
            al += L[a][k] * (w0[k] - wm1[k]);
            ar += L[a][k] * (wp1[k] - w0[k]);
            ac += L[a][k] * (0.5 * (wp1[k] - wm1[k]));
        }
        da[a] = mc_limit(al, ar, ac);
    }
    for (int k = 0; k < 7; k++) {
        double s = 0.0;
        for (int a = 0; a < 7; a++) s += R[k][a] * da[a];
        dw[k] = s;
    }
}

static double clip(double x, double a, double b)
{
    double lo = dmin(a, b), hi = dmax(a, b);
    return dmin(dmax(x, lo), hi);
}

void orc_recon_cell(int recon, int trace, const double *w5flat, const double bn5[5], double gam, double dtdx,
                    double wm[7], double wp[7])
{
    const double (*w5)[7] = (const double (*)[7])w5flat;
    const double *w0 = w5[2];
    if (recon == PLM_PRIM) {
        /* primitive-variable PLM (no characteristic projection), MC limiter */
        for (int k = 0; k < 7; k++) {
            double d = mc_limit(w0[k] - w5[1][k], w5[3][k] - w0[k], 0.5 * (w5[3][k] - w5[1][k]));
            wm[k] = w0[k] - 0.5 * d;
            wp[k] = w0[k] + 0.5 * d;
        }
        return;
    }
    double lam[7], R[7][7], L[7][7];
    eigen7(w0[0], w0[1], gam * w0[4] / w0[0], bn5[2], w0[5], w0[6], lam, R, L);
    double pl[7], pr[7];   /* characteristic deviations of the face values from the centre */
    if (recon == PLM) {
        for (int a = 0; a < 7; a++) {
            double al = 0.0, ar = 0.0, ac = 0.0;
            for (int k = 0; k < 7; k++) {
                al += L[a][k] * (w0[k] - w5[1][k]);
                ar += L[a][k] * (w5[3][k] - w0[k]);
                ac += L[a][k] * (0.5 * (w5[3][k] - w5[1][k]));
            }
            double d = mc_limit(al, ar, ac);
            pl[a] = -0.5 * d;
            pr[a] = 0.5 * d;
        }
    } else {
        /* PPM (Colella & Woodward 1984): interface values from the limited  */
        /* slopes of the three cells, bounded by the adjacent cell values,   */
        /* then monotonised per characteristic field.                         */
        double dwm[7], dw0[7], dwp[7], fm[7], fp[7];
        char_slope(w5[0], w5[1], w5[2], bn5[1], gam, dwm);
        char_slope(w5[1], w5[2], w5[3], bn5[2], gam, dw0);
        char_slope(w5[2], w5[3], w5[4], bn5[3], gam, dwp);
        for (int k = 0; k < 7; k++) {
            double vm = 0.5 * (w5[1][k] + w0[k]) - (dw0[k] - dwm[k]) / 6.0;
            double vp = 0.5 * (w0[k] + w5[3][k]) - (dwp[k] - dw0[k]) / 6.0;
            fm[k] = clip(vm, w5[1][k], w0[k]) - w0[k];
            fp[k] = clip(vp, w0[k], w5[3][k]) - w0[k];
        }
        for (int a = 0; a < 7; a++) {
            double l = 0.0, r = 0.0;
            for (int k = 0; k < 7; k++) { l += L[a][k] * fm[k]; r += L[a][k] * fp[k]; }
            if (l * r >= 0.0) { l = 0.0; r = 0.0; }
            else {
                double dlt = r - l, a6 = -3.0 * (l + r);
                if (dlt * a6 > dlt * dlt) l = -2.0 * r;
                else if (-dlt * dlt > dlt * a6) r = -2.0 * l;
            }
            pl[a] = l;
            pr[a] = r;
        }
    }
    double fl[7], fr[7];
    if (!trace) {
        for (int a = 0; a < 7; a++) { fl[a] = pl[a]; fr[a] = pr[a]; }
    } else {
        /* CTU characteristic tracing to t + dt/2: each wave's face value is */
        /* the parabola (line, for PLM) averaged over the part of the cell   */
        /* its characteristic sweeps in dt/2; waves moving away from a face  */
        /* take the domain of the fastest wave moving towards it.            */
        double smax = dmax(lam[6], 0.0) * dtdx;
        double smin = dmin(lam[0], 0.0) * dtdx;
        for (int a = 0; a < 7; a++) {
            double dlt = pr[a] - pl[a], a6 = -3.0 * (pl[a] + pr[a]);
            double sp = lam[a] > 0.0 ? lam[a] * dtdx : smax;
            double sm = lam[a] < 0.0 ? lam[a] * dtdx : smin;
            fr[a] = pr[a] - 0.5 * sp * (dlt - (1.0 - 2.0 / 3.0 * sp) * a6);
            fl[a] = pl[a] - 0.5 * sm * (dlt + (1.0 + 2.0 / 3.0 * sm) * a6);
        }
    }
    for (int k = 0; k < 7; k++) {
        double sl = 0.0, sr = 0.0;
        for (int a = 0; a < 7; a++) { sl += R[k][a] * fl[a]; sr += R[k][a] * fr[a]; }
        wm[k] = w0[k] + sl;
        wp[k] = w0[k] + sr;
        if (!trace) {
            wm[k] = clip(wm[k], w5[1][k], w0[k]);
            wp[k] = clip(wp[k], w0[k], w5[3][k]);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Whole-grid helpers                                                        */
/* ------------------------------------------------------------------------ */

/* cell-centred primitives (rho, vx, vy, vz, P, Bx, By, Bz) from U and the   */
/* face B; B at the cell centre is the mean of its two faces (Fig. 1).       */
/* With a pressure floor (g->pfloor > 0, not part of the paper's scheme; the  */
/* option used for blast and low-beta stress states) P below the floor is     */
/* replaced by the floor; when e_raise is given (the energy array U + 4n, at  */
/* the start of a step) the total energy of such a cell is raised by         */
/* (pfloor - P)/(gamma - 1) so that the state carries P = pfloor.  Returns     */
/* the number of floored cells.                                               */
static long prim_floor(const grid_t *g, const double *U, const double *B, double *W, double *e_raise)
{
    long n = g->n, cnt = 0;
#pragma omp parallel for schedule(static) reduction(+:cnt)
    for (long c = 0; c < n; c++) {
        double rho = U[c];
        double vx = U[n + c] / rho, vy = U[2 * n + c] / rho, vz = U[3 * n + c] / rho;
        double bx = 0.5 * (B[c] + B[shift(g, c, 0, 1)]);
        double by = 0.5 * (B[n + c] + B[n + shift(g, c, 1, 1)]);
        double bz = 0.5 * (B[2 * n + c] + B[2 * n + shift(g, c, 2, 1)]);
        double p = (g->gam - 1.0) * (U[4 * n + c] - 0.5 * rho * (vx * vx + vy * vy + vz * vz)
                                     - 0.5 * (bx * bx + by * by + bz * bz));
        if (g->pfloor > 0.0 && p < g->pfloor) {
            if (e_raise) {
                e_raise[c] = e_raise[c] + (g->pfloor - p) / (g->gam - 1.0);
                cnt++;
            }
            p = g->pfloor;
        }
        W[c] = rho; W[n + c] = vx; W[2 * n + c] = vy; W[3 * n + c] = vz;
        W[4 * n + c] = p; W[5 * n + c] = bx; W[6 * n + c] = by; W[7 * n + c] = bz;
    }
    return cnt;
}

static void prim_all(const grid_t *g, const double *U, const double *B, double *W)
{
    prim_floor(g, U, B, W, NULL);
}

/* sweep-frame primitive vector of cell c for a sweep along d */
static void rot_prim(const grid_t *g, const double *W, long c, int d, double w[7], double *bn)
{
    long n = g->n;
    int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    w[0] = W[c];
    w[1] = W[(1 + d) * n + c];
    w[2] = W[(1 + t1) * n + c];
    w[3] = W[(1 + t2) * n + c];
    w[4] = W[4 * n + c];
    w[5] = W[(5 + t1) * n + c];
    w[6] = W[(5 + t2) * n + c];
    *bn = W[(5 + d) * n + c];
}

/* Eq. 10: conservative update U -= h * div F (F[d][7][n] in sweep frames).  */
/* Along an outflow axis the last cell's upper face is not stored: its flux  */
/* is the Riemann flux between the last cell and its zero-gradient ghost,    */
/* taken from Fout[d][7][n] at the last cell when given (CTU), else formed   */
/* here (VL): both face states are then the last cell's state Wst (the       */
/* stage's primitives), since the limited slope against a copied ghost is    */
/* zero for PLM and PPM, with the normal field of the last face.             */
static int is_last(const grid_t *g, long c, int d)
{
    if (d == 0) return (int)(c % g->nx) == g->nx - 1;
    if (d == 1) return (int)((c / g->nx) % g->ny) == g->ny - 1;
    return (int)(c / ((long)g->nx * g->ny)) == g->nz - 1;
}

static void fv_update(const grid_t *g, double h, const double *Usrc, const double *F, double *Udst,
                      const double *Wst, const double *Bst, int riemann, const double *Fout)
{
    long n = g->n;
    double r = h / g->dx;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; c++) {
        double du[5] = {0, 0, 0, 0, 0};
        for (int d = 0; d < 3; d++) {
            int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
            long cp = shift(g, c, d, 1);
            const double *Fd = F + (long)d * 7 * n;
            double df[7];
            if ((g->bc >> d & 1) && is_last(g, c, d)) {
                double fu[7];
                if (Fout) {
                    for (int k = 0; k < 7; k++) fu[k] = Fout[((long)d * 7 + k) * n + c];
                } else {
                    double w[7], bdum;
                    rot_prim(g, Wst, c, d, w, &bdum);
                    orc_riemann(riemann, w, w, Bst[d * n + c], g->gam, fu);
                }
                for (int k = 0; k < 7; k++) df[k] = fu[k] - Fd[k * n + c];
            } else {
                for (int k = 0; k < 7; k++) df[k] = Fd[k * n + cp] - Fd[k * n + c];
            }
            du[0] += df[0];
            du[1 + d] += df[1];
            du[1 + t1] += df[2];
            du[1 + t2] += df[3];
            du[4] += df[4];
        }
        for (int f = 0; f < 5; f++) Udst[f * n + c] = Usrc[f * n + c] - r * du[f];
    }
}

/* CTU step 3 / VL step 2: edge electric field from the face fields of the   */
/* Riemann fluxes, the cell-centre reference E = -v x B and the face mass    */
/* fluxes (upwinded corner average, Gardiner & Stone 2005).                   */
/* E_c lives on the edge along c at the lower (a,b) corner of cell (a,b),    */
/* a = c+1, b = c+2 (cyclic): Ez at (i-1/2,j-1/2,k), Ex at (i,j-1/2,k-1/2),   */
/* Ey at (i-1/2,j,k-1/2).                                                     */
static double upw(double f, double xm, double xp)
{
    if (f > 0.0) return xm;
    if (f < 0.0) return xp;
    return 0.5 * (xm + xp);
}

static void edge_emf(const grid_t *g, const double *F, const double *W, double *E)
{
    long n = g->n;
    for (int c = 0; c < 3; c++) {
        int a = (c + 1) % 3, b = (c + 2) % 3;
        const double *Fa = F + (long)a * 7 * n;   /* sweep along a: t1 = b, t2 = c */
        const double *Fb = F + (long)b * 7 * n;   /* sweep along b: t1 = c, t2 = a */
#pragma omp parallel for schedule(static)
        for (long q = 0; q < n; q++) {
            long c11 = q;                        /* cell (a=i,   b=j)   */
            long c01 = shift(g, q, a, -1);       /* cell (a=i-1, b=j)   */
            long c10 = shift(g, q, b, -1);       /* cell (a=i,   b=j-1) */
            long c00 = shift(g, c01, b, -1);     /* cell (a=i-1, b=j-1) */
            /* E_c on the a-faces (a = i-1/2) at b = j-1, j: -F_a[B_b] */
            double ea0 = -Fa[5 * n + c10], ea1 = -Fa[5 * n + c11];
            /* E_c on the b-faces (b = j-1/2) at a = i-1, i: +F_b[B_a] */
            double eb0 = Fb[6 * n + c01], eb1 = Fb[6 * n + c11];
            double fa0 = Fa[c10], fa1 = Fa[c11];  /* mass fluxes */
            double fb0 = Fb[c01], fb1 = Fb[c11];
            double cc[4];
            long cells[4] = {c00, c10, c01, c11};
            for (int m = 0; m < 4; m++) {
                long s = cells[m];
                double va = W[(1 + a) * n + s], vb = W[(1 + b) * n + s];
                double ba = W[(5 + a) * n + s], bb = W[(5 + b) * n + s];
                cc[m] = -(va * bb - vb * ba);
            }
            double cc00 = cc[0], cc10 = cc[1], cc01 = cc[2], cc11 = cc[3];
            double hib = upw(fa1, cc01 - eb0, cc11 - eb1);
            double lob = upw(fa0, eb0 - cc00, eb1 - cc10);
            double hia = upw(fb1, cc10 - ea0, cc11 - ea1);
            double loa = upw(fb0, ea0 - cc00, ea1 - cc01);
            E[c * n + q] = 0.25 * (ea0 + ea1 + eb0 + eb1) + 0.25 * (lob - hib) + 0.25 * (loa - hia);
        }
    }
}

/* Eq. 13: CT update of the face fields, B_d -= h * (curl E)_d on faces      */
static void ct_update(const grid_t *g, double h, const double *Bsrc, const double *E, double *Bdst)
{
    long n = g->n;
    double r = h / g->dx;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; c++) {
        for (int d = 0; d < 3; d++) {
            int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
            double curl = (E[t2 * n + shift(g, c, t1, 1)] - E[t2 * n + c])
                        - (E[t1 * n + shift(g, c, t2, 1)] - E[t1 * n + c]);
            Bdst[d * n + c] = Bsrc[d * n + c] - r * curl;
        }
    }
}

/* reconstruct + Riemann along every axis: F[d][7][n], face c - 1/2 e_d.     */
/* ws, bs: optional per-direction face states (CTU); when given, the flux    */
/* uses them instead of reconstructing from W.                               */
static long fluxes(const grid_t *g, int recon, int riemann, int first_order, int trace, double dt,
                   const double *W, const double *Bface, double *F,
                   double *WMs, double *WPs)
{
    long n = g->n;
    long nfb = 0;
    for (int d = 0; d < 3; d++) {
        double *WMd = WMs ? WMs + (long)d * 7 * n : NULL;
        double *WPd = WPs ? WPs + (long)d * 7 * n : NULL;
        double *tmpM = NULL, *tmpP = NULL;
        if (!first_order) {
            tmpM = WMd ? WMd : (double *)malloc(sizeof(double) * 7 * n);
            tmpP = WPd ? WPd : (double *)malloc(sizeof(double) * 7 * n);
#pragma omp parallel for schedule(static)
            for (long c = 0; c < n; c++) {
                double w5[5][7], b5[5], wm[7], wp[7];
                for (int m = 0; m < 5; m++) rot_prim(g, W, shift(g, c, d, m - 2), d, w5[m], &b5[m]);
                orc_recon_cell(recon, trace, &w5[0][0], b5, g->gam, dt / g->dx, wm, wp);
                for (int k = 0; k < 7; k++) { tmpM[k * n + c] = wm[k]; tmpP[k * n + c] = wp[k]; }
            }
            ORC_STAGE("reconstruction");
        }
        double *Fd = F + (long)d * 7 * n;
#pragma omp parallel for schedule(static) reduction(+ : nfb)
        for (long c = 0; c < n; c++) {
            long cl = shift(g, c, d, -1);
            double wl[7], wr[7], f[7], bdum;
            if (first_order) {
                rot_prim(g, W, cl, d, wl, &bdum);
                rot_prim(g, W, c, d, wr, &bdum);
            } else {
                for (int k = 0; k < 7; k++) { wl[k] = tmpP[k * n + cl]; wr[k] = tmpM[k * n + c]; }
            }
            nfb += orc_riemann(riemann, wl, wr, Bface[d * n + c], g->gam, f);
            for (int k = 0; k < 7; k++) Fd[k * n + c] = f[k];
        }
        ORC_STAGE(first_order ? "riemann_predictor" : "riemann_corrector");
        if (!first_order) {
            if (!WMd) free(tmpM);
            if (!WPd) free(tmpP);
        }
    }
    return nfb;
}

/* ------------------------------------------------------------------------ */
/* One step of the VL scheme (Sec. 3.2, VL steps 1-7).                       */
/* ------------------------------------------------------------------------ */
static long step_vl(const grid_t *g, int recon, int riemann, double dt, double *U, double *B, long *nfloor)
{
    long n = g->n;
    double *W = (double *)malloc(sizeof(double) * 8 * n);
    double *F = (double *)malloc(sizeof(double) * 21 * n);
    double *E = (double *)malloc(sizeof(double) * 3 * n);
    double *Uh = (double *)malloc(sizeof(double) * 5 * n);
    double *Bh = (double *)malloc(sizeof(double) * 3 * n);
    long nfb = 0;
    /* steps 1-3: first-order fluxes with face B_n, edge E, half update */
    *nfloor += prim_floor(g, U, B, W, U + 4 * n);
    ORC_STAGE("primitives");
    nfb += fluxes(g, recon, riemann, 1, 0, dt, W, B, F, NULL, NULL);
    edge_emf(g, F, W, E);
    ORC_STAGE("edge_emf");
    fv_update(g, 0.5 * dt, U, F, Uh, W, B, riemann, NULL);
    ct_update(g, 0.5 * dt, B, E, Bh);
    ORC_STAGE("half_update");
    /* steps 4-7: reconstruct at the half step, Riemann, edge E, full update */
    prim_all(g, Uh, Bh, W);
    ORC_STAGE("primitives");
    nfb += fluxes(g, recon, riemann, 0, 0, dt, W, Bh, F, NULL, NULL);
    edge_emf(g, F, W, E);
    ORC_STAGE("edge_emf");
    fv_update(g, dt, U, F, U, W, Bh, riemann, NULL);
    ct_update(g, dt, B, E, B);
    ORC_STAGE("full_update");
    free(W); free(F); free(E); free(Uh); free(Bh);
    return nfb;
}

/* ------------------------------------------------------------------------ */
/* One step of the CTU scheme (Sec. 3.2, CTU steps 1-8).                     */
/* ------------------------------------------------------------------------ */

/* CTU step 5 for one traced state: the state w of cell s on a d-face (from  */
/* WM or WP), as 8 conserved components with B_n of cell s at its centre,    */
/* receives -dt/2 times the divergence of the other two axes' stage-1 fluxes */
/* across cell s, and goes back to primitives.  Along an outflow axis e the  */
/* last cell's upper e-face flux is Fo1[e] at that cell.                     */
static void ctu_corrected(const grid_t *g, int d, long s, const double *wsrc, const double *W, const double *F,
                          const double *Fo1, double hdt, double wout[7])
{
    long n = g->n;
    double gam = g->gam;
    int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    double w[7];
    for (int k = 0; k < 7; k++) w[k] = wsrc[k * n + s];
    /* global-frame conserved vector: rho, M(3), e, B(3) */
    double bcc[3] = {W[5 * n + s], W[6 * n + s], W[7 * n + s]};
    double q[8];
    double bglob[3];
    bglob[d] = bcc[d]; bglob[t1] = w[5]; bglob[t2] = w[6];
    double vglob[3];
    vglob[d] = w[1]; vglob[t1] = w[2]; vglob[t2] = w[3];
    q[0] = w[0];
    for (int m = 0; m < 3; m++) q[1 + m] = w[0] * vglob[m];
    q[4] = w[4] / (gam - 1.0) + 0.5 * w[0] * (vglob[0] * vglob[0] + vglob[1] * vglob[1] + vglob[2] * vglob[2])
           + 0.5 * (bglob[0] * bglob[0] + bglob[1] * bglob[1] + bglob[2] * bglob[2]);
    for (int m = 0; m < 3; m++) q[5 + m] = bglob[m];
    int axes[2] = {t1, t2};
    for (int m = 0; m < 2; m++) {
        int e = axes[m];
        int e1 = (e + 1) % 3, e2 = (e + 2) % 3;
        const double *Fe = F + (long)e * 7 * n;
        double df[7];
        if ((g->bc >> e & 1) && is_last(g, s, e)) {
            for (int k = 0; k < 7; k++) df[k] = Fo1[((long)e * 7 + k) * n + s] - Fe[k * n + s];
        } else {
            long sp = shift(g, s, e, 1);
            for (int k = 0; k < 7; k++) df[k] = Fe[k * n + sp] - Fe[k * n + s];
        }
        double r = hdt / g->dx;
        q[0] -= r * df[0];
        q[1 + e] -= r * df[1];
        q[1 + e1] -= r * df[2];
        q[1 + e2] -= r * df[3];
        q[4] -= r * df[4];
        q[5 + e1] -= r * df[5];
        q[5 + e2] -= r * df[6];
    }
    double rho = q[0];
    double vx = q[1] / rho, vy = q[2] / rho, vz = q[3] / rho;
    double p = (gam - 1.0) * (q[4] - 0.5 * rho * (vx * vx + vy * vy + vz * vz)
                              - 0.5 * (q[5] * q[5] + q[6] * q[6] + q[7] * q[7]));
    double vg[3] = {vx, vy, vz};
    wout[0] = rho;
    wout[1] = vg[d];
    wout[2] = vg[t1];
    wout[3] = vg[t2];
    wout[4] = p;
    wout[5] = q[5 + t1];
    wout[6] = q[5 + t2];
}

/* outflow: the flux through the outer (upper) face of each last cell along   */
/* each outflow axis, into Fo[d][7][n] at that cell.  The ghost beyond it is  */
/* the last cell itself (reading of the zero-gradient rule used throughout),  */
/* so the face states are the cell's own upper (plus) and lower (minus)       */
/* states of the stage; stage 2 corrects both as in step 5.                   */
static long ctu_outer_fluxes(const grid_t *g, int riemann, const double *WM, const double *WP, const double *Bn,
                             const double *W, const double *F, const double *Fo1, double hdt, double *Fo)
{
    long n = g->n, nfb = 0;
    for (int d = 0; d < 3; d++) {
        if (!(g->bc >> d & 1)) continue;
        const double *WMd = WM + (long)d * 7 * n, *WPd = WP + (long)d * 7 * n;
#pragma omp parallel for schedule(static) reduction(+ : nfb)
        for (long c = 0; c < n; c++) {
            if (!is_last(g, c, d)) continue;
            double wl[7], wr[7], f[7];
            if (F) {
                ctu_corrected(g, d, c, WPd, W, F, Fo1, hdt, wl);
                ctu_corrected(g, d, c, WMd, W, F, Fo1, hdt, wr);
            } else {
                for (int k = 0; k < 7; k++) { wl[k] = WPd[k * n + c]; wr[k] = WMd[k * n + c]; }
            }
            nfb += orc_riemann(riemann, wl, wr, Bn[d * n + c], g->gam, f);
            for (int k = 0; k < 7; k++) Fo[((long)d * 7 + k) * n + c] = f[k];
        }
    }
    return nfb;
}

static long step_ctu(const grid_t *g, int recon, int riemann, double dt, double *U, double *B, long *nfloor)
{
    long n = g->n;
    double gam = g->gam;
    double *W = (double *)malloc(sizeof(double) * 8 * n);
    double *F = (double *)malloc(sizeof(double) * 21 * n);
    double *F2 = (double *)malloc(sizeof(double) * 21 * n);
    double *E = (double *)malloc(sizeof(double) * 3 * n);
    double *Uh = (double *)malloc(sizeof(double) * 5 * n);
    double *Bh = (double *)malloc(sizeof(double) * 3 * n);
    double *WM = (double *)malloc(sizeof(double) * 21 * n);
    double *WP = (double *)malloc(sizeof(double) * 21 * n);
    long nfb = 0;
    double hdt = 0.5 * dt;
    /* step 1: traced face states at t+dt/2 along every axis */
    *nfloor += prim_floor(g, U, B, W, U + 4 * n);
    ORC_STAGE("primitives");
    {
        /* fill WM/WP via the reconstruction pass, then add the source terms  */
        /* the 1-D system leaves out when dB_n/dn != 0: in primitive form     */
        /* S = (0, B/rho, -(gamma-1) v.B, v_t1, v_t2) * dB_n/dn, times dt/2.   */
        for (int d = 0; d < 3; d++) {
            double *WMd = WM + (long)d * 7 * n, *WPd = WP + (long)d * 7 * n;
#pragma omp parallel for schedule(static)
            for (long c = 0; c < n; c++) {
                double w5[5][7], b5[5], wm[7], wp[7];
                for (int m = 0; m < 5; m++) rot_prim(g, W, shift(g, c, d, m - 2), d, w5[m], &b5[m]);
                orc_recon_cell(recon, 1, &w5[0][0], b5, gam, dt / g->dx, wm, wp);
                double dbn = (B[d * n + shift(g, c, d, 1)] - B[d * n + c]) / g->dx;
                const double *w = w5[2];
                double bn = b5[2];
                double vb = w[1] * bn + w[2] * w[5] + w[3] * w[6];
                double src[7] = {0.0, bn / w[0], w[5] / w[0], w[6] / w[0], -(gam - 1.0) * vb, w[2], w[3]};
                for (int k = 0; k < 7; k++) {
                    WMd[k * n + c] = wm[k] + hdt * src[k] * dbn;
                    WPd[k * n + c] = wp[k] + hdt * src[k] * dbn;
                }
            }
        }
    }
    ORC_STAGE("reconstruction_tracing");
    /* step 2: Riemann fluxes of the traced states with the face B_n at t^n */
    for (int d = 0; d < 3; d++) {
        double *Fd = F + (long)d * 7 * n;
        const double *WMd = WM + (long)d * 7 * n, *WPd = WP + (long)d * 7 * n;
#pragma omp parallel for schedule(static) reduction(+ : nfb)
        for (long c = 0; c < n; c++) {
            long cl = shift(g, c, d, -1);
            double wl[7], wr[7], f[7];
            for (int k = 0; k < 7; k++) { wl[k] = WPd[k * n + cl]; wr[k] = WMd[k * n + c]; }
            nfb += orc_riemann(riemann, wl, wr, B[d * n + c], gam, f);
            for (int k = 0; k < 7; k++) Fd[k * n + c] = f[k];
        }
    }
    ORC_STAGE("riemann_predictor");
    /* outflow: the stage-1 fluxes through the outer faces */
    double *Fo1 = NULL, *Fo2 = NULL;
    if (g->bc) {
        Fo1 = (double *)calloc((size_t)21 * n, sizeof(double));
        Fo2 = (double *)calloc((size_t)21 * n, sizeof(double));
        nfb += ctu_outer_fluxes(g, riemann, WM, WP, B, W, NULL, NULL, hdt, Fo1);
    }
    /* step 3: edge E from these fluxes and the cell-centre E at t^n */
    edge_emf(g, F, W, E);
    ORC_STAGE("edge_emf");
    /* step 4: dt/2 CT update of face B and conservative update of U */
    ct_update(g, hdt, B, E, Bh);
    fv_update(g, hdt, U, F, Uh, NULL, NULL, riemann, Fo1);
    ORC_STAGE("half_update");
    /* step 5: transverse flux-gradient correction of the traced states     */
    /* (ctu_corrected), and step 6: Riemann with the half-step face B_n     */
    for (int d = 0; d < 3; d++) {
        double *Fd = F2 + (long)d * 7 * n;
        const double *WMd = WM + (long)d * 7 * n, *WPd = WP + (long)d * 7 * n;
#pragma omp parallel for schedule(static) reduction(+ : nfb)
        for (long c = 0; c < n; c++) {
            double wface[2][7];
            ctu_corrected(g, d, shift(g, c, d, -1), WPd, W, F, Fo1, hdt, wface[0]);
            ctu_corrected(g, d, c, WMd, W, F, Fo1, hdt, wface[1]);
            ORC_STAGE("transverse_correction");
            double f[7];
            nfb += orc_riemann(riemann, wface[0], wface[1], Bh[d * n + c], gam, f);
            for (int k = 0; k < 7; k++) Fd[k * n + c] = f[k];
            ORC_STAGE("riemann_corrector");
        }
    }
    if (g->bc) nfb += ctu_outer_fluxes(g, riemann, WM, WP, Bh, W, F, Fo1, hdt, Fo2);
    /* step 7: edge E from the corrected fluxes and the half-step cell state */
    prim_all(g, Uh, Bh, W);
    ORC_STAGE("primitives");
    edge_emf(g, F2, W, E);
    ORC_STAGE("edge_emf");
    /* step 8: full update */
    fv_update(g, dt, U, F2, U, NULL, NULL, riemann, Fo2);
    ct_update(g, dt, B, E, B);
    ORC_STAGE("full_update");
    free(Fo1); free(Fo2);
    free(W); free(F); free(F2); free(E); free(Uh); free(Bh); free(WM); free(WP);
    return nfb;
}

/* ------------------------------------------------------------------------ */
/* Exported whole-grid entry points                                          */
/* ------------------------------------------------------------------------ */

/* advance U, B in place by dt with a pressure floor (0 = none) and the     */
/* boundary mask bc (bit d: outflow along axis d); returns the number of     */
/* Roe->HLLE fallbacks, the floored cells in *nfloor                         */
long orc_step_full(int nx, int ny, int nz, double dx, double gam, int integrator, int recon, int riemann,
                   double dt, double pfloor, int bc, double *U, double *B, long *nfloor)
{
    grid_t g = {nx, ny, nz, (long)nx * ny * nz, dx, gam, pfloor, bc};
    *nfloor = 0;
    if (integrator == CTU) return step_ctu(&g, recon, riemann, dt, U, B, nfloor);
    return step_vl(&g, recon, riemann, dt, U, B, nfloor);
}

long orc_step_floor(int nx, int ny, int nz, double dx, double gam, int integrator, int recon, int riemann,
                    double dt, double pfloor, double *U, double *B, long *nfloor)
{
    return orc_step_full(nx, ny, nz, dx, gam, integrator, recon, riemann, dt, pfloor, 0, U, B, nfloor);
}

/* advance U, B in place by dt; returns the number of Roe->HLLE fallbacks */
long orc_step(int nx, int ny, int nz, double dx, double gam, int integrator, int recon, int riemann,
              double dt, double *U, double *B)
{
    long nf = 0;
    return orc_step_full(nx, ny, nz, dx, gam, integrator, recon, riemann, dt, 0.0, 0, U, B, &nf);
}

/* CFL time step (Sec. 3.2): cfl * dx / max over cells and axes of |v_d| + c_f,d, */
/* with the pressure floor of the step applied to P (0 = none) and the boundary   */
/* mask of the step (the cell-centre field of the last cell along an outflow axis) */
double orc_cfl_dt_full(int nx, int ny, int nz, double dx, double gam, double cfl, double pfloor, int bc,
                       const double *U, const double *B)
{
    grid_t g = {nx, ny, nz, (long)nx * ny * nz, dx, gam, pfloor, bc};
    long n = g.n;
    double *W = (double *)malloc(sizeof(double) * 8 * n);
    prim_all(&g, U, B, W);
    double smax = 0.0;
    for (long c = 0; c < n; c++) {
        double rho = W[c], p = W[4 * n + c];
        double a2 = gam * p / rho;
        for (int d = 0; d < 3; d++) {
            int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
            double cf = fast_speed(rho, a2, W[(5 + d) * n + c], W[(5 + t1) * n + c], W[(5 + t2) * n + c]);
            double s = fabs(W[(1 + d) * n + c]) + cf;
            if (s > smax) smax = s;
        }
    }
    free(W);
    return cfl * dx / smax;
}

double orc_cfl_dt_floor(int nx, int ny, int nz, double dx, double gam, double cfl, double pfloor, const double *U,
                        const double *B)
{
    return orc_cfl_dt_full(nx, ny, nz, dx, gam, cfl, pfloor, 0, U, B);
}

double orc_cfl_dt(int nx, int ny, int nz, double dx, double gam, double cfl, const double *U, const double *B)
{
    return orc_cfl_dt_full(nx, ny, nz, dx, gam, cfl, 0.0, 0, U, B);
}

/* Eq. 16 times dx: max_c |sum_d (B_d(c+e_d) - B_d(c))|, and B_rms of the     */
/* cell-centred field                                                         */
void orc_divB_bc(int nx, int ny, int nz, int bc, const double *B, double *maxabs, double *brms)
{
    grid_t g = {nx, ny, nz, (long)nx * ny * nz, 1.0, 0.0, 0.0, bc};
    long n = g.n;
    double m = 0.0, s2 = 0.0;
    for (long c = 0; c < n; c++) {
        double dv = 0.0, b2 = 0.0;
        for (int d = 0; d < 3; d++) {
            double bp = B[d * n + shift(&g, c, d, 1)], b0 = B[d * n + c];
            dv += bp - b0;
            double bc_ = 0.5 * (bp + b0);
            b2 += bc_ * bc_;
        }
        if (fabs(dv) > m) m = fabs(dv);
        s2 += b2;
    }
    *maxabs = m;
    *brms = sqrt(s2 / (double)n);
}

void orc_divB(int nx, int ny, int nz, const double *B, double *maxabs, double *brms)
{
    orc_divB_bc(nx, ny, nz, 0, B, maxabs, brms);
}

/* sums of rho, Mx, My, Mz, e over cells and of Bx, By, Bz over faces */
void orc_sums(int nx, int ny, int nz, const double *U, const double *B, double out[8])
{
    long n = (long)nx * ny * nz;
    for (int f = 0; f < 8; f++) {
        const double *a = f < 5 ? U + (long)f * n : B + (long)(f - 5) * n;
        double s = 0.0;
        for (long c = 0; c < n; c++) s += a[c];
        out[f] = s;
    }
}

/* cell-centred primitives, exported for diagnostics */
void orc_prim_bc(int nx, int ny, int nz, double gam, int bc, const double *U, const double *B, double *W)
{
    grid_t g = {nx, ny, nz, (long)nx * ny * nz, 1.0, gam, 0.0, bc};
    prim_all(&g, U, B, W);
}

void orc_prim(int nx, int ny, int nz, double gam, const double *U, const double *B, double *W)
{
    orc_prim_bc(nx, ny, nz, gam, 0, U, B, W);
}

/* ------------------------------------------------------------------------ */
/* Diagnostics of Sec. 4.3 / 4.5: current density J = curl B on the cell    */
/* edges (Stokes' theorem on the four faces around an edge), and the         */
/* energy integrals E_T, U_B, U_V of Sec. 4.5.                               */
/* ------------------------------------------------------------------------ */

/* dx times J on the edges: J_x at (i, j-1/2, k-1/2), J_y at (i-1/2, j,       */
/* k-1/2), J_z at (i-1/2, j-1/2, k), the layout of the edge E fields:         */
/*   dx J_a = (B_c(c) - B_c(c - e_b)) - (B_b(c) - B_b(c - e_c)),  b = a+1, c = a+2 */
void orc_edge_current(int nx, int ny, int nz, const double *B, double *J)
{
    grid_t g = {nx, ny, nz, (long)nx * ny * nz, 1.0, 0.0};
    long n = g.n;
    for (long c = 0; c < n; c++) {
        for (int a = 0; a < 3; a++) {
            int b = (a + 1) % 3, cc = (a + 2) % 3;
            J[a * n + c] = (B[cc * n + c] - B[cc * n + shift(&g, c, b, -1)])
                         - (B[b * n + c] - B[b * n + shift(&g, c, cc, -1)]);
        }
    }
}

/* out[0] E_T   = sum e dx^3                                                  */
/* out[1] U_B   = sum over faces B_f^2/2 dx^3 (the face-based magnetic energy) */
/* out[2] U_V   = sum |M|^2/(2 rho) dx^3                                      */
/* out[3] max over cells of dx |J_cc| / |B_cc|; J_cc the mean of the four     */
/*        edges of the cell along each axis, B_cc the mean of its two faces    */
/* out[4] number of cells with dx |J_cc| / |B_cc| > thr (the refinement test  */
/*        |J|/|B| > thr/dx of Sec. 4.3 and 4.5)                                */
/* out[5] max over cells of |J_cc|                                            */
void orc_energies(int nx, int ny, int nz, double dx, const double *U, const double *B, double thr, double out[6])
{
    grid_t g = {nx, ny, nz, (long)nx * ny * nz, dx, 0.0};
    long n = g.n;
    double *J = (double *)malloc(sizeof(double) * 3 * n);
    orc_edge_current(nx, ny, nz, B, J);
    double et = 0.0, ub = 0.0, uv = 0.0, rmax = 0.0, jmax = 0.0, cnt = 0.0;
    for (long c = 0; c < n; c++) {
        et += U[4 * n + c];
        double m2 = U[n + c] * U[n + c] + U[2 * n + c] * U[2 * n + c] + U[3 * n + c] * U[3 * n + c];
        uv += 0.5 * m2 / U[c];
        double jc[3], bc[3];
        for (int a = 0; a < 3; a++) {
            int b = (a + 1) % 3, cc = (a + 2) % 3;
            ub += 0.5 * B[a * n + c] * B[a * n + c];
            long cb = shift(&g, c, b, 1), ccc = shift(&g, c, cc, 1), cbc = shift(&g, cb, cc, 1);
            jc[a] = 0.25 * (J[a * n + c] + J[a * n + cb] + J[a * n + ccc] + J[a * n + cbc]);
            bc[a] = 0.5 * (B[a * n + c] + B[a * n + shift(&g, c, a, 1)]);
        }
        double jm = sqrt(jc[0] * jc[0] + jc[1] * jc[1] + jc[2] * jc[2]);
        double bm = sqrt(bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
        double r = jm / bm;
        if (r > rmax) rmax = r;
        if (r > thr) cnt += 1.0;
        if (jm > jmax) jmax = jm;
    }
    free(J);
    double v = dx * dx * dx;
    out[0] = et * v;
    out[1] = ub * v;
    out[2] = uv * v;
    out[3] = rmax;
    out[4] = cnt;
    out[5] = jmax / dx;
}

/* threads of the OpenMP loops (the CPU-baseline timings run 1 and all);    */
/* returns the count in effect                                              */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
