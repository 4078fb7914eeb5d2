// Per-event kinematics shared by the diagram kernels (mg_kernels.cu, and
// mg_big.cu for the processes whose state lives in HBM): momentum sums of
// every gluon subset, 1/P^2 and the top-line propagators, computed once per
// event and reused by all helicities; the helicity index of a work unit; the
// unit-modulus jamp coefficients.
#pragma once
#include "mg_dirac.cuh"

namespace mg {

template <int NG>
struct Kin {
    static constexpr int NPAR = NG + 2;
    static constexpr int NS = 1 << NG;
    double P[NPAR][4];   // momenta as given
    double K[NS][4];     // sum of incoming momenta of the gluons in subset S
    double IP2[NS];      // 1 / K_S^2
    double QP[NS][4];    // top-line momentum after absorbing S from ubar: p3 - K_S
    cx DP[NS];           // 1 / (QP^2 - m^2 + i m w)
    double QS[NS][4];    // top-line momentum after absorbing S from v: K_S - p4
    cx DS[NS];           // 1 / (QS^2 - m^2 + i m w)
};

__device__ __forceinline__ cx cinv(double a, double b) {
    const double d = 1.0 / fma(a, a, b * b);
    return mk(a * d, -b * d);
}

template <int NG>
__device__ void kinematics(Kin<NG> &k, const double *__restrict__ p, double mt, double wt) {
    constexpr int NPAR = NG + 2, NS = 1 << NG;
#pragma unroll
    for (int i = 0; i < NPAR; i++)
#pragma unroll
        for (int m = 0; m < 4; m++) k.P[i][m] = __ldg(p + 4 * i + m);
    double Kg[NG][4];
#pragma unroll
    for (int g = 0; g < NG; g++) {
        const int ip = (g < 2) ? g : g + 2;
        const double sg = (g < 2) ? 1.0 : -1.0;
#pragma unroll
        for (int m = 0; m < 4; m++) Kg[g][m] = sg * k.P[ip][m];
    }
    const double m2 = mt * mt, mw = mt * wt;
    for (int m = 0; m < 4; m++) k.K[0][m] = 0.0;
    k.IP2[0] = 0.0;
    for (int S = 1; S < NS; S++) {
        const int low = __ffs(S) - 1;
        const int rest = S & (S - 1);
        for (int m = 0; m < 4; m++) k.K[S][m] = k.K[rest][m] + Kg[low][m];
        const double *K = k.K[S];
        const double k2 = K[0] * K[0] - K[1] * K[1] - K[2] * K[2] - K[3] * K[3];
        k.IP2[S] = rest ? 1.0 / k2 : 0.0;
        double q2 = 0.0, s2 = 0.0;
        for (int m = 0; m < 4; m++) {
            k.QP[S][m] = k.P[2][m] - K[m];
            k.QS[S][m] = K[m] - k.P[3][m];
            const double g = (m == 0) ? 1.0 : -1.0;
            q2 += g * k.QP[S][m] * k.QP[S][m];
            s2 += g * k.QS[S][m] * k.QS[S][m];
        }
        k.DP[S] = cinv(q2 - m2, mw);
        k.DS[S] = cinv(s2 - m2, mw);
    }
}

// Full helicity index of gluon configuration g (bit j = helicity of gluon j,
// gluons in particle order) and top/antitop helicity bits bt, btb.
template <int NG>
__device__ __forceinline__ int helicity_index(int g, int bt, int btb) {
    constexpr int NPAR = NG + 2;
    int h = (bt << (NPAR - 1 - 2)) | (btb << (NPAR - 1 - 3));
#pragma unroll
    for (int j = 0; j < NG; j++) {
        const int ip = (j < 2) ? j : j + 2;
        h |= ((g >> j) & 1) << (NPAR - 1 - ip);
    }
    return h;
}

// unit-modulus coefficient {+1, -1, +i, -i}[code] times a
__device__ __forceinline__ cx unit_times(int code, cx a) {
    switch (code & 3) {
        case 0: return a;
        case 1: return mk(-a.r, -a.i);
        case 2: return mk(-a.i, a.r);
        default: return mk(a.i, -a.r);
    }
}

}  // namespace mg
