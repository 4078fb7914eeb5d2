/*
 * CPU oracle for the leading-order matrix element of g g -> t t~ + (n-2) g.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of the benchmark load this library.  It shares no code, header or table
 * with the CUDA path.
 *
 * What it computes (plain definition, FP64, built -ffp-contract=off):
 *   |M|^2 averaged = (1/IDEN) sum_h  g^(2n) sum_{s,t} conj(A_s) C_st A_t
 * with A_s the colour-ordered amplitude of ordering s of the n gluons along
 * the top line, C_st = Tr((T^s)^dagger T^t) the colour matrix (exact rational,
 * built by oracle/color.py and passed in), and h all helicity combinations.
 * This is the colour-flow/quadratic-form structure of the paper's colour sum
 * (Sec. 3.3, Eq. "jcj": J^H C J with C real symmetric), evaluated here by a
 * different algorithm than the Feynman-diagram method: the colour-ordered
 * amplitudes come from Berends-Giele recursion, which the paper
 * (Sec. 4.5) names as the better approach for many gluons.
 *
 * Conventions (textbook QCD, metric +---, Tr(t^a t^b) = delta^ab / 2):
 *   quark-gluon vertex  i g gamma^mu t^a
 *   3-gluon vertex      g f^abc [g^mn (k-p)^r + g^nr (p-q)^m + g^rm (q-k)^n]
 *   4-gluon vertex      -i g^2 [f f (gg - gg) x 3]
 *   gluon propagator    -i g_mn / k^2  (Feynman gauge)
 *   top propagator      i (qslash + m) / (q^2 - m^2 + i m Gamma)
 * Expanding f^abc t^c = -i [t^a, t^b] gives the colour-ordered rules used in
 * the recursion (all momenta incoming, gluon sub-words X,Y,Z in order):
 *   3-vertex  -i V(k_X, k_Y, q)
 *   4-vertex  i (2 g^{XZ} g^{Y.} - g^{XY} g^{Z.} - g^{YZ} g^{X.})
 * External states: gluons are circular polarisation vectors with zero time
 * component in the frame the momenta are given in (incoming eps, outgoing
 * eps*); tops are helicity eigenstates ubar(p3, h3), v(p4, h4) in the chiral
 * (Weyl) representation.  A helicity index h has bit (npar-1-i) set when
 * particle i has positive helicity; particle order is g1 g2 t t~ g5 ... .
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define MAXG 8            /* up to 8 gluons */
#define NPMAX (MAXG + 2)

/* Minkowski product of complex 4-vectors (no conjugation). */
static cplx mdot(const cplx *a, const cplx *b) {
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}
static double mdotr(const double *a, const double *b) {
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}
static cplx mdotrc(const double *a, const cplx *b) {
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

/* gamma^mu in the chiral representation, gamma^mu[row][col]. */
static cplx GAM[4][4][4];
static int gam_ready = 0;

static void init_gamma(void) {
    if (gam_ready) return;
    memset(GAM, 0, sizeof(GAM));
    /* sigma^k */
    cplx sig[4][2][2];
    memset(sig, 0, sizeof(sig));
    sig[0][0][0] = 1; sig[0][1][1] = 1;              /* identity */
    sig[1][0][1] = 1; sig[1][1][0] = 1;
    sig[2][0][1] = -I; sig[2][1][0] = I;
    sig[3][0][0] = 1; sig[3][1][1] = -1;
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) {
            /* gamma^0 = [[0, 1], [1, 0]] */
            GAM[0][i][2 + j] = sig[0][i][j];
            GAM[0][2 + i][j] = sig[0][i][j];
            for (int k = 1; k <= 3; k++) {
                /* gamma^k = [[0, sigma^k], [-sigma^k, 0]] */
                GAM[k][i][2 + j] = sig[k][i][j];
                GAM[k][2 + i][j] = -sig[k][i][j];
            }
        }
    gam_ready = 1;
}

/* M = a_slash = gamma^0 a^0 - gamma^k a^k  (a has upper indices). */
static void slash(const cplx *a, cplx M[4][4]) {
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++)
            M[r][c] = GAM[0][r][c] * a[0] - GAM[1][r][c] * a[1] - GAM[2][r][c] * a[2] -
                      GAM[3][r][c] * a[3];
}

/* row spinor times matrix */
static void rowmul(const cplx *r, cplx M[4][4], cplx *out) {
    cplx t[4];
    for (int c = 0; c < 4; c++) {
        t[c] = 0;
        for (int k = 0; k < 4; k++) t[c] += r[k] * M[k][c];
    }
    memcpy(out, t, sizeof(t));
}

/* Two-component helicity eigenvectors chi_{+-}(p_hat) of p_hat . sigma. */
static void chi(const double *p, int h, cplx out[2]) {
    double pa = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    double th = (pa > 0) ? acos(fmax(-1.0, fmin(1.0, p[3] / pa))) : 0.0;
    double ph = atan2(p[2], p[1]);
    double c = cos(0.5 * th), s = sin(0.5 * th);
    if (h > 0) {
        out[0] = c;
        out[1] = cexp(I * ph) * s;
    } else {
        out[0] = -cexp(-I * ph) * s;
        out[1] = c;
    }
}

/* u(p, h): (sqrt(E - h|p|) chi_h, sqrt(E + h|p|) chi_h) */
static void spinor_u(const double *p, int h, cplx u[4]) {
    double pa = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    cplx x[2];
    chi(p, h, x);
    double a = sqrt(fmax(0.0, p[0] - h * pa)), b = sqrt(fmax(0.0, p[0] + h * pa));
    u[0] = a * x[0]; u[1] = a * x[1]; u[2] = b * x[0]; u[3] = b * x[1];
}

/* v(p, h) for an antiparticle of helicity h:
 * (sqrt(E + h|p|) chi_{-h}, -sqrt(E - h|p|) chi_{-h}) */
static void spinor_v(const double *p, int h, cplx v[4]) {
    double pa = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    cplx x[2];
    chi(p, -h, x);
    double a = sqrt(fmax(0.0, p[0] + h * pa)), b = sqrt(fmax(0.0, p[0] - h * pa));
    v[0] = a * x[0]; v[1] = a * x[1]; v[2] = -b * x[0]; v[3] = -b * x[1];
}

/* ubar = u^dagger gamma^0 */
static void spinor_ubar(const double *p, int h, cplx ub[4]) {
    cplx u[4];
    spinor_u(p, h, u);
    for (int c = 0; c < 4; c++) {
        ub[c] = 0;
        for (int k = 0; k < 4; k++) ub[c] += conj(u[k]) * GAM[0][k][c];
    }
}

/* Circular polarisation eps(k, lam), lam = +-1, eps^0 = 0:
 * eps = (-lam e1 - i e2) / sqrt2,
 * e1 = (0, cos th cos ph, cos th sin ph, -sin th), e2 = (0, -sin ph, cos ph, 0). */
static void polvec(const double *p, int lam, cplx e[4]) {
    double pa = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    double th = acos(fmax(-1.0, fmin(1.0, p[3] / pa)));
    double ph = atan2(p[2], p[1]);
    double e1[4] = {0, cos(th) * cos(ph), cos(th) * sin(ph), -sin(th)};
    double e2[4] = {0, -sin(ph), cos(ph), 0};
    for (int m = 0; m < 4; m++) e[m] = (-lam * e1[m] - I * e2[m]) / sqrt(2.0);
}

/* Colour-ordered 3-vertex contracted with J1, J2 (momenta k1, k2 incoming,
 * third leg q = -(k1+k2)):
 * V^r = (J1.J2)(k1-k2)^r + J2^r (k1+2k2).J1 - J1^r (2k1+k2).J2 */
static void v3(const cplx *J1, const double *k1, const cplx *J2, const double *k2, cplx *out) {
    double a[4], b[4], d[4];
    for (int m = 0; m < 4; m++) {
        d[m] = k1[m] - k2[m];
        a[m] = k1[m] + 2 * k2[m];
        b[m] = 2 * k1[m] + k2[m];
    }
    cplx j12 = mdot(J1, J2), s2 = mdotrc(a, J1), s1 = mdotrc(b, J2);
    for (int m = 0; m < 4; m++) out[m] = j12 * d[m] + J2[m] * s2 - J1[m] * s1;
}

/* Colour-ordered 4-vertex (without the factor i):
 * 2 (J1.J3) J2 - (J1.J2) J3 - (J2.J3) J1 */
static void v4(const cplx *J1, const cplx *J2, const cplx *J3, cplx *out) {
    cplx a = mdot(J1, J3), b = mdot(J1, J2), c = mdot(J2, J3);
    for (int m = 0; m < 4; m++) out[m] = 2 * a * J2[m] - b * J3[m] - c * J1[m];
}

typedef struct {
    double mt, wt;     /* top mass, top width */
} params_t;

/* Colour-ordered amplitude A(3_t, g_sig[0..n-1], 4_tbar) by Berends-Giele.
 * eps[i], kin[i]: polarisation vector and incoming momentum of gluon i
 * (i indexes the n gluons in particle order), ub: ubar(p3), v: v(p4). */
static cplx bg_amplitude(int n, const int *sig, cplx eps[][4], double kin[][4], const cplx *ub,
                         const cplx *v, const double *p3, const params_t *par) {
    cplx J[MAXG][MAXG][4];
    double K[MAXG][MAXG][4];
    for (int len = 1; len <= n; len++) {
        for (int a = 0; a + len - 1 < n; a++) {
            int b = a + len - 1;
            if (len == 1) {
                memcpy(J[a][a], eps[sig[a]], sizeof(cplx) * 4);
                memcpy(K[a][a], kin[sig[a]], sizeof(double) * 4);
                continue;
            }
            for (int m = 0; m < 4; m++) K[a][b][m] = K[a][a][m] + K[a + 1][b][m];
            cplx acc[4] = {0, 0, 0, 0}, t[4];
            /* 3-vertex splits: current = (-i/P^2)(-i) V3 = -V3/P^2 */
            for (int m = a; m < b; m++) {
                v3(J[a][m], K[a][m], J[m + 1][b], K[m + 1][b], t);
                for (int c = 0; c < 4; c++) acc[c] -= t[c];
            }
            /* 4-vertex splits: current = (-i/P^2)(i) V4 = V4/P^2 */
            for (int m = a; m < b; m++)
                for (int l = m + 1; l < b; l++) {
                    v4(J[a][m], J[m + 1][l], J[l + 1][b], t);
                    for (int c = 0; c < 4; c++) acc[c] += t[c];
                }
            double P2 = mdotr(K[a][b], K[a][b]);
            for (int c = 0; c < 4; c++) J[a][b][c] = acc[c] / P2;
        }
    }
    /* top line from ubar(p3): U[j] absorbed gluons sig[0..j-1] */
    cplx U[MAXG + 1][4];
    memcpy(U[0], ub, sizeof(cplx) * 4);
    cplx M[4][4], t[4];
    for (int j = 1; j <= n; j++) {
        for (int c = 0; c < 4; c++) U[j][c] = 0;
        for (int m = 0; m < j; m++) {
            slash(J[m][j - 1], M); /* vertex i gamma.J */
            rowmul(U[m], M, t);
            for (int c = 0; c < 4; c++) U[j][c] += I * t[c];
        }
        if (j == n) break;
        /* propagator i (qslash + m)/(q^2 - m^2 + i m w), q = p3 - K[0][j-1] */
        cplx q[4];
        double qr[4];
        for (int m = 0; m < 4; m++) {
            qr[m] = p3[m] - K[0][j - 1][m];
            q[m] = qr[m];
        }
        slash(q, M);
        for (int r = 0; r < 4; r++) M[r][r] += par->mt;
        rowmul(U[j], M, t);
        cplx den = mdotr(qr, qr) - par->mt * par->mt + I * par->mt * par->wt;
        for (int c = 0; c < 4; c++) U[j][c] = I * t[c] / den;
    }
    cplx amp = 0;
    for (int c = 0; c < 4; c++) amp += U[n][c] * v[c];
    return amp;
}

/* External states of one event for helicity index h.  gauge_leg >= 0
 * replaces that gluon's polarisation by its momentum (Ward-identity test). */
static void externals(int n, const double *mom, int h, int gauge_leg, cplx eps[][4],
                      double kin[][4], cplx *ub, cplx *v) {
    int npar = n + 2;
    for (int g = 0; g < n; g++) {
        int ip = (g < 2) ? g : g + 2; /* particle index of gluon g */
        const double *p = mom + 4 * ip;
        int lam = ((h >> (npar - 1 - ip)) & 1) ? 1 : -1;
        int incoming = (ip < 2);
        for (int m = 0; m < 4; m++) kin[g][m] = incoming ? p[m] : -p[m];
        if (g == gauge_leg) {
            for (int m = 0; m < 4; m++) eps[g][m] = p[m];
        } else {
            polvec(p, lam, eps[g]);
            if (!incoming)
                for (int m = 0; m < 4; m++) eps[g][m] = conj(eps[g][m]);
        }
    }
    int h3 = ((h >> (npar - 1 - 2)) & 1) ? 1 : -1;
    int h4 = ((h >> (npar - 1 - 3)) & 1) ? 1 : -1;
    spinor_ubar(mom + 8, h3, ub);
    spinor_v(mom + 12, h4, v);
}

/* ------------------------------------------------------------------ API -- */

/* All colour-ordered amplitudes of one event and helicity.
 * perms: [ncolor][n] gluon indices (0..n-1 in particle order g1 g2 g5 ...).
 * amps_out: [ncolor] complex as (re, im) pairs.  Couplings are not included. */
int oracle_amplitudes(int n, const double *mom, int h, int gauge_leg, const double *par_in,
                      int ncolor, const int *perms, double *amps_out) {
    if (n < 2 || n > MAXG) return -1;
    init_gamma();
    params_t par = {par_in[0], par_in[1]};
    cplx eps[MAXG][4], ub[4], v[4];
    double kin[MAXG][4];
    externals(n, mom, h, gauge_leg, eps, kin, ub, v);
    for (int s = 0; s < ncolor; s++) {
        cplx a = bg_amplitude(n, perms + s * n, eps, kin, ub, v, mom + 8, &par);
        amps_out[2 * s] = creal(a);
        amps_out[2 * s + 1] = cimag(a);
    }
    return 0;
}

/* Matrix elements for nevt events.
 * n: number of gluons (incoming included); mom: [nevt][n+2][4];
 * par_in: {mt, wt, gs}; cnum: [ncolor][ncolor] colour-matrix numerators,
 * cden: common denominator; perms: [ncolor][n]; iden: averaging factor;
 * hel_mask: [2^(n+2)] (NULL = all helicities);
 * me_out: [nevt]; me_hel_out: [nevt][2^(n+2)] per-helicity |M_h|^2 (optional,
 * already divided by iden).  nthreads <= 0 uses the OpenMP default. */
int oracle_me(int n, const double *mom, int64_t nevt, const double *par_in, const int64_t *cnum,
              int64_t cden, int ncolor, const int *perms, double iden, const uint8_t *hel_mask,
              double *me_out, double *me_hel_out, int nthreads) {
    if (n < 2 || n > MAXG || nevt < 0) return -1;
    init_gamma();
    int npar = n + 2, nhel = 1 << npar;
    params_t par = {par_in[0], par_in[1]};
    double g2n = pow(par_in[2], 2 * n);
    double *C = (double *)malloc(sizeof(double) * (size_t)ncolor * ncolor);
    if (!C) return -2;
    for (size_t i = 0; i < (size_t)ncolor * ncolor; i++) C[i] = (double)cnum[i] / (double)cden;
    /* |M_h|^2 of every (event, helicity) pair first, in parallel over the
     * pairs (a handful of events of the large processes still spreads over
     * all threads), then each event's sum over h in order */
    const int64_t npairs = nevt * (int64_t)nhel;
    double *mh_all = (double *)malloc(sizeof(double) * (size_t)(npairs > 0 ? npairs : 1));
    if (!mh_all) {
        free(C);
        return -2;
    }
    int status = 0;
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel num_threads(nt)
#endif
    {
        cplx *A = (cplx *)malloc(sizeof(cplx) * ncolor);
        if (!A) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            status = -2;
        }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t q = 0; q < npairs; q++) {
            if (!A) continue;
            const int64_t e = q / nhel;
            const int h = (int)(q % nhel);
            const double *p = mom + (size_t)e * npar * 4;
            double mh = 0;
            if (!hel_mask || hel_mask[h]) {
                cplx eps[MAXG][4], ub[4], v[4];
                double kin[MAXG][4];
                externals(n, p, h, -1, eps, kin, ub, v);
                for (int s = 0; s < ncolor; s++)
                    A[s] = bg_amplitude(n, perms + s * n, eps, kin, ub, v, p + 8, &par);
                double acc = 0;
                for (int s = 0; s < ncolor; s++) {
                    cplx z = 0;
                    for (int t = 0; t < ncolor; t++) z += C[(size_t)s * ncolor + t] * A[t];
                    acc += creal(conj(A[s]) * z);
                }
                mh = g2n * acc / iden;
            }
            mh_all[q] = mh;
        }
        free(A);
    }
    for (int64_t e = 0; e < nevt; e++) {
        double tot = 0;
        for (int h = 0; h < nhel; h++) {
            const double mh = mh_all[e * nhel + h];
            if (me_hel_out) me_hel_out[(size_t)e * nhel + h] = mh;
            tot += mh;
        }
        me_out[e] = tot;
    }
    free(mh_all);
    free(C);
    return status;
}

/* Number of OpenMP threads the library would use. */
int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* External states of one event and helicity index, for the oracle's
 * single-diagram evaluation (oracle/sde.py): eps_out [n][4] polarisation
 * vectors (incoming eps, outgoing eps*), kin_out [n][4] incoming momenta of
 * the gluons, ub_out [4] = ubar(p3), v_out [4] = v(p4); complex values as
 * (re, im) pairs.  Same conventions as the Berends-Giele amplitudes above. */
int oracle_externals(int n, const double *mom, int h, double *eps_out, double *kin_out,
                     double *ub_out, double *v_out) {
    if (n < 2 || n > MAXG) return -1;
    init_gamma();
    cplx eps[MAXG][4], ub[4], v[4];
    double kin[MAXG][4];
    externals(n, mom, h, -1, eps, kin, ub, v);
    for (int g = 0; g < n; g++)
        for (int m = 0; m < 4; m++) {
            eps_out[8 * g + 2 * m] = creal(eps[g][m]);
            eps_out[8 * g + 2 * m + 1] = cimag(eps[g][m]);
            kin_out[4 * g + m] = kin[g][m];
        }
    for (int c = 0; c < 4; c++) {
        ub_out[2 * c] = creal(ub[c]);
        ub_out[2 * c + 1] = cimag(ub[c]);
        v_out[2 * c] = creal(v[c]);
        v_out[2 * c + 1] = cimag(v[c]);
    }
    return 0;
}
