// Device building blocks of the Feynman-diagram calculation: external
// wavefunctions (the roles of the paper's vxxxxx / ixxxxx / oxxxxx, Sec. 2.2),
// gluon currents through the 3- and 4-gluon vertices, top-line
// wavefunctions with propagators, and amplitude contractions (the roles of
// the ALOHA routines VVV1P0_1, FFV1_0, ... named in Sec. 2.2).
//
// Dirac algebra in the chiral representation, 2x2 blocks:
//   gamma^mu = [[0, sigma^mu], [sigmabar^mu, 0]],
//   aslash   = [[0, A], [B, 0]],  A = a.sigma = a^0 - a.sigma_vec,
//                                 B = a.sigmabar = a^0 + a.sigma_vec.
// Spinors are 4 complex components (L pair, R pair); Lorentz vectors have
// upper indices; metric (+,-,-,-).  All arithmetic is FP64.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace mg {

struct cx {
    double r, i;
};

__device__ __forceinline__ cx mk(double r, double i) { return cx{r, i}; }
__device__ __forceinline__ cx operator+(cx a, cx b) { return cx{a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ cx operator-(cx a, cx b) { return cx{a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ cx operator-(cx a) { return cx{-a.r, -a.i}; }
__device__ __forceinline__ cx operator*(cx a, cx b) {
    return cx{fma(a.r, b.r, -a.i * b.i), fma(a.r, b.i, a.i * b.r)};
}
__device__ __forceinline__ cx operator*(double s, cx a) { return cx{s * a.r, s * a.i}; }
// a*b + c
__device__ __forceinline__ cx cfma(cx a, cx b, cx c) {
    return cx{fma(a.r, b.r, fma(-a.i, b.i, c.r)), fma(a.r, b.i, fma(a.i, b.r, c.i))};
}
// s*a + c with real s
__device__ __forceinline__ cx rfma(double s, cx a, cx c) { return cx{fma(s, a.r, c.r), fma(s, a.i, c.i)}; }

// Minkowski products
__device__ __forceinline__ cx mdot(const cx *a, const cx *b) {
    cx t = a[0] * b[0];
    t = cfma(-a[1], b[1], t);
    t = cfma(-a[2], b[2], t);
    return cfma(-a[3], b[3], t);
}
__device__ __forceinline__ cx mdot_r(const double *k, const cx *b) {
    cx t = k[0] * b[0];
    t = rfma(-k[1], b[1], t);
    t = rfma(-k[2], b[2], t);
    return rfma(-k[3], b[3], t);
}

// ------------------------------------------------------- external states --

// Circular polarisation of a massless gluon with momentum p and helicity
// lam = +-1: eps = (-lam e1 - i e2)/sqrt(2) with eps^0 = 0 in the frame of the
// momenta, (e1, e2, p_hat) right-handed:
//   e1 = (0, px pz/(|p| pt), py pz/(|p| pt), -pt/|p|), e2 = (0, -py/pt, px/pt, 0)
// (pt = 0: e1 = (0, sign pz, 0, 0), e2 = (0, 0, 1, 0)).  Outgoing gluons
// take the complex conjugate.
__device__ __forceinline__ void ext_gluon(const double *p, int lam, bool incoming, cx *e) {
    const double px = p[1], py = p[2], pz = p[3];
    const double pt2 = px * px + py * py;
    const double pt = sqrt(pt2);
    const double pa = sqrt(pt2 + pz * pz);
    double e1x, e1y, e1z, e2x, e2y;
    if (pt > 0.0) {
        const double c = pz / (pa * pt);
        e1x = px * c;
        e1y = py * c;
        e1z = -pt / pa;
        e2x = -py / pt;
        e2y = px / pt;
    } else {
        e1x = (pz >= 0.0) ? 1.0 : -1.0;
        e1y = 0.0;
        e1z = 0.0;
        e2x = 0.0;
        e2y = 1.0;
    }
    const double h = 0.70710678118654752440;  // 1/sqrt(2)
    const double sr = -lam * h;                // real part factor
    const double si = incoming ? -h : h;       // imaginary part factor (conj if outgoing)
    e[0] = mk(0.0, 0.0);
    e[1] = mk(sr * e1x, si * e2x);
    e[2] = mk(sr * e1y, si * e2y);
    e[3] = mk(sr * e1z, 0.0);
}

// Two-component helicity eigenvector of p_hat.sigma for helicity sign h:
//   chi_+ = (sqrt(|p|+pz), (px + i py)/sqrt(|p|+pz)) / sqrt(2|p|)
//   chi_- = ((-px + i py)/sqrt(|p|+pz), sqrt(|p|+pz)) / sqrt(2|p|)
// with |p|+pz = pt^2/(|p|-pz) for pz < 0 (no cancellation).
__device__ __forceinline__ void helicity_2spinor(const double *p, int h, cx *x) {
    const double px = p[1], py = p[2], pz = p[3];
    const double pt2 = px * px + py * py;
    const double pa = sqrt(pt2 + pz * pz);
    const double a = (pz >= 0.0) ? pa + pz : pt2 / (pa - pz);
    if (a > 0.0) {
        const double sa = sqrt(a), nrm = 1.0 / sqrt(2.0 * pa), isa = nrm / sa;
        if (h > 0) {
            x[0] = mk(sa * nrm, 0.0);
            x[1] = mk(px * isa, py * isa);
        } else {
            x[0] = mk(-px * isa, py * isa);
            x[1] = mk(sa * nrm, 0.0);
        }
    } else {  // along -z
        if (h > 0) {
            x[0] = mk(0.0, 0.0);
            x[1] = mk(1.0, 0.0);
        } else {
            x[0] = mk(-1.0, 0.0);
            x[1] = mk(0.0, 0.0);
        }
    }
}

// ubar(p, h) of an outgoing top: u = (sqrt(E - h|p|) chi_h, sqrt(E + h|p|) chi_h),
// ubar = u^dagger gamma^0 = (u3*, u4*, u1*, u2*).
__device__ __forceinline__ void ext_ubar(const double *p, int h, cx *ub) {
    cx x[2];
    helicity_2spinor(p, h, x);
    const double pa = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    const double wm = sqrt(fmax(p[0] - h * pa, 0.0)), wp = sqrt(fmax(p[0] + h * pa, 0.0));
    ub[0] = mk(wp * x[0].r, -wp * x[0].i);
    ub[1] = mk(wp * x[1].r, -wp * x[1].i);
    ub[2] = mk(wm * x[0].r, -wm * x[0].i);
    ub[3] = mk(wm * x[1].r, -wm * x[1].i);
}

// v(p, h) of an outgoing antitop of helicity h:
// v = (sqrt(E + h|p|) chi_{-h}, -sqrt(E - h|p|) chi_{-h}).
__device__ __forceinline__ void ext_v(const double *p, int h, cx *v) {
    cx x[2];
    helicity_2spinor(p, -h, x);
    const double pa = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
    const double wp = sqrt(fmax(p[0] + h * pa, 0.0)), wm = sqrt(fmax(p[0] - h * pa, 0.0));
    v[0] = wp * x[0];
    v[1] = wp * x[1];
    v[2] = (-wm) * x[0];
    v[3] = (-wm) * x[1];
}

// ------------------------------------------------------------- vertices --

// Gluon current through the 3-gluon vertex, divided by its propagator
// denominator: J = ( (J1.J2)(K1-K2) + J2 (K1+2K2).J1 - J1 (2K1+K2).J2 ) / P^2
// (K1, K2 incoming momenta of the two sub-currents, P = K1 + K2).
__device__ __forceinline__ void vvv_current(const cx *J1, const double *K1, const cx *J2,
                                            const double *K2, double invP2, cx *out) {
    double a[4], b[4], d[4];
#pragma unroll
    for (int m = 0; m < 4; m++) {
        d[m] = K1[m] - K2[m];
        a[m] = fma(2.0, K2[m], K1[m]);
        b[m] = fma(2.0, K1[m], K2[m]);
    }
    const cx j12 = invP2 * mdot(J1, J2);
    const cx s2 = invP2 * mdot_r(a, J1);
    const cx s1 = -(invP2 * mdot_r(b, J2));
#pragma unroll
    for (int m = 0; m < 4; m++) out[m] = cfma(s1, J1[m], cfma(s2, J2[m], d[m] * j12));
}

// The three 4-gluon-vertex structures for sub-currents X, Y, Z:
//   L1 = (X.Z) Y - (Y.Z) X,  L2 = (X.Y) Z - (Y.Z) X,  L3 = (X.Y) Z - (X.Z) Y,
// each divided by P^2.
__device__ __forceinline__ void vvvv_currents(const cx *X, const cx *Y, const cx *Z, double invP2,
                                              cx *o1, cx *o2, cx *o3) {
    const cx xy = invP2 * mdot(X, Y), xz = invP2 * mdot(X, Z), yz = invP2 * mdot(Y, Z);
    const cx myz = -yz, mxz = -xz;
#pragma unroll
    for (int m = 0; m < 4; m++) {
        o1[m] = cfma(xz, Y[m], myz * X[m]);
        o2[m] = cfma(xy, Z[m], myz * X[m]);
        o3[m] = cfma(xy, Z[m], mxz * Y[m]);
    }
}

// Blocks of Jslash: jp = J0+J3, jm = J0-J3, t = J1 + i J2, tc = J1 - i J2;
// A = [[jm, -tc], [-t, jp]], B = [[jp, tc], [t, jm]].
struct Slash {
    cx jp, jm, t, tc;
};
__device__ __forceinline__ Slash slash_blocks(const cx *J) {
    Slash s;
    s.jp = J[0] + J[3];
    s.jm = J[0] - J[3];
    s.t = mk(J[1].r - J[2].i, J[1].i + J[2].r);
    s.tc = mk(J[1].r + J[2].i, J[1].i - J[2].r);
    return s;
}

// row spinor times Jslash: (u3,u4).B , (u1,u2).A
__device__ __forceinline__ void row_slash(const cx *u, const Slash &s, cx *o) {
    o[0] = cfma(u[2], s.jp, u[3] * s.t);
    o[1] = cfma(u[2], s.tc, u[3] * s.jm);
    o[2] = cfma(u[0], s.jm, -(u[1] * s.t));
    o[3] = cfma(u[1], s.jp, -(u[0] * s.tc));
}

// Jslash times column spinor: A (v3,v4), B (v1,v2)
__device__ __forceinline__ void slash_col(const Slash &s, const cx *v, cx *o) {
    o[0] = cfma(s.jm, v[2], -(s.tc * v[3]));
    o[1] = cfma(s.jp, v[3], -(s.t * v[2]));
    o[2] = cfma(s.jp, v[0], s.tc * v[1]);
    o[3] = cfma(s.t, v[0], s.jm * v[1]);
}

// complex a times (q1 + i*sgn*q2) for real q1, q2
__device__ __forceinline__ cx mul_s(cx a, double q1, double q2) {
    return mk(fma(a.r, q1, -a.i * q2), fma(a.r, q2, a.i * q1));
}

// row t times (qslash + m), q real:
//   ( m t1 + qp t3 + s t4,  m t2 + sc t3 + qm t4,
//     qm t1 - s t2 + m t3, -sc t1 + qp t2 + m t4 ),  s = q1 + i q2
__device__ __forceinline__ void row_qm(const cx *t, const double *q, double m, cx *o) {
    const double qp = q[0] + q[3], qm = q[0] - q[3];
    o[0] = rfma(m, t[0], rfma(qp, t[2], mul_s(t[3], q[1], q[2])));
    o[1] = rfma(m, t[1], rfma(qm, t[3], mul_s(t[2], q[1], -q[2])));
    o[2] = rfma(m, t[2], rfma(qm, t[0], -mul_s(t[1], q[1], q[2])));
    o[3] = rfma(m, t[3], rfma(qp, t[1], -mul_s(t[0], q[1], -q[2])));
}

// (qslash + m) times column y:
//   ( m y1 + qm y3 - sc y4,  m y2 - s y3 + qp y4,
//     qp y1 + sc y2 + m y3,  s y1 + qm y2 + m y4 )
__device__ __forceinline__ void qm_col(const double *q, double m, const cx *y, cx *o) {
    const double qp = q[0] + q[3], qm = q[0] - q[3];
    o[0] = rfma(m, y[0], rfma(qm, y[2], -mul_s(y[3], q[1], -q[2])));
    o[1] = rfma(m, y[1], rfma(qp, y[3], -mul_s(y[2], q[1], q[2])));
    o[2] = rfma(m, y[2], rfma(qp, y[0], mul_s(y[1], q[1], -q[2])));
    o[3] = rfma(m, y[3], rfma(qm, y[1], mul_s(y[0], q[1], q[2])));
}

// Gamma^mu = U gamma^mu V (4 complex components, upper index)
__device__ __forceinline__ void bilinear(const cx *u, const cx *v, cx *g) {
    const cx a11 = u[0] * v[2], a12 = u[0] * v[3], a21 = u[1] * v[2], a22 = u[1] * v[3];
    const cx b11 = u[2] * v[0], b12 = u[2] * v[1], b21 = u[3] * v[0], b22 = u[3] * v[1];
    g[0] = (a11 + a22) + (b11 + b22);
    g[1] = (a12 + a21) - (b12 + b21);
    const cx w = (a21 - a12) - (b21 - b12);
    g[2] = mk(-w.i, w.r);  // i * w
    g[3] = (a11 - a22) - (b11 - b22);
}

__device__ __forceinline__ cx sdot(const cx *x, const cx *v) {
    cx t = x[0] * v[0];
    t = cfma(x[1], v[1], t);
    t = cfma(x[2], v[2], t);
    return cfma(x[3], v[3], t);
}

}  // namespace mg
