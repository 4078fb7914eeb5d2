// Processes whose per-thread state does not fit in local memory: g g -> t t~
// + 5 g (810k ops, 12527 gluon + 3989 top-line slots, 8505 accumulators and
// 5040 colour flows: about 2 MB per work unit, above the 512 KB a thread
// may hold in local memory).  The paper's CUDA build of this process failed
// to link (its generated code is too large); here the same table-driven
// program runs with its state in HBM, which the arithmetic still dominates:
// about 150 FP64 flops per 200 bytes of state moved, right of the FP64 ridge
// of a GB300.
//
// Four kernels per chunk of events:
//   k_kin_big       the kinematic tables of each event (momentum sums of the
//                   gluon subsets, propagator denominators), once per event.
//   k_sigmakin_big  one thread per work item (event, gluon-helicity
//                   configuration with its four top helicities), persistent
//                   over the items.  Wavefunction slots and accumulators live
//                   in a slot-major, thread-interleaved scratch (element i of
//                   thread t at scratch[i * T + t], so a warp's accesses are
//                   coalesced); the jamps accumulate directly into the FP64
//                   colour-major rows of the colour sum, row
//                   r = 2 (v * nipad + item) + re/im, colour c at c * R + r
//                   (real and imaginary part of a jamp side by side).  Jamp
//                   updates and the sums of colour-factor groups are FP64
//                   reductions performed at L2 (red.global.add.f64): the
//                   thread never waits for a jamp row, and these additions
//                   (about a fifth of the FP64 instructions) leave the FP64
//                   pipe; measured 0.490 -> 0.632 of the FP64 peak.
//   k_colour_big    the colour sum J^H C J (Sec. 3.3, Eq. "jcj") of every
//                   row as a tiled FP64 quadratic form over the block upper
//                   triangle of D*C (off-diagonal 64 x 64 blocks doubled, the
//                   paper's triangular colour sum at tile granularity):
//                   qpart[I][r] = sum_{n in tile I} V_rn sum_{k >= 64 I} Cb_nk V_rk.
//   k_event_sum_big per event, the sum over its items, good helicity
//                   combinations, real/imaginary rows and tiles in a fixed
//                   order (and |M_h|^2 per helicity for the filter; the
//                   per-event alpha_s factor and channel weight of the
//                   extras).
// In mixed precision k_rows_to_bf16 turns the rows into BF16 pieces and the
// block-triangular tensor-core kernel of mg_colorsum_tc.cu replaces
// k_colour_big; k_flow_weights_big gives the per-flow weights of the extras.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mg_dirac.cuh"
#include "mg_internal.h"
#include "mg_kin.cuh"

using namespace mg;

namespace {

constexpr int BIG_NG = 7;
constexpr int BIG_BLOCK = 128;
constexpr int CT = 64;   // colour tile (n and k) of the quadratic form
constexpr int CK = 16;   // k chunk per shared-memory stage
constexpr int RT = 64;   // rows per tile

// slot-major, thread-interleaved state; p already offset by the thread
struct Strided {
    double2 *p;
    long long T;
    __device__ __forceinline__ cx ld(long long i) const {
        const double2 v = p[i * T];
        return mk(v.x, v.y);
    }
    __device__ __forceinline__ void st(long long i, cx c) const { p[i * T] = make_double2(c.r, c.i); }
    __device__ __forceinline__ void ld4(long long i0, cx *o) const {
#pragma unroll
        for (int m = 0; m < 4; m++) o[m] = ld(i0 + m);
    }
    __device__ __forceinline__ void st4(long long i0, const cx *o) const {
#pragma unroll
        for (int m = 0; m < 4; m++) st(i0 + m, o[m]);
    }
};

__device__ __forceinline__ void red_add(double *p, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed(double2 *p, cx v) {
    asm volatile("st.relaxed.gpu.global.v2.f64 [%0], {%1, %2};" ::"l"(p), "d"(v.r), "d"(v.i) : "memory");
}

__device__ __forceinline__ cx ld_relaxed(const double2 *p) {
    double r, i;
    asm volatile("ld.relaxed.gpu.global.v2.f64 {%0, %1}, [%2];" : "=d"(r), "=d"(i) : "l"(p) : "memory");
    return mk(r, i);
}

__device__ __forceinline__ void prefetch_l2(const double2 *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// slot s of a pool with `per` elements per slot
__device__ __forceinline__ void prefetch_slot(const Strided &P, int per, int s) {
    for (int m = 0; m < per; m++) prefetch_l2(P.p + (long long)(per * s + m) * P.T);
}

// The wavefunctions an op will read (same field meaning as run_item).
__device__ __forceinline__ void prefetch_inputs(const int4 &a, const int4 &b, const Strided &WG,
                                                const Strided &WF, const Strided &ACC) {
    switch (a.x) {
        case MG_OP_V3:
            prefetch_slot(WG, 4, a.z);
            prefetch_slot(WG, 4, a.w);
            break;
        case MG_OP_V4:
            prefetch_slot(WG, 4, b.x);
            prefetch_slot(WG, 4, b.y);
            prefetch_slot(WG, 4, b.z);
            break;
        case MG_OP_FPRE:
        case MG_OP_FSUF:
        case MG_OP_XROW:
            prefetch_slot(WG, 4, a.w);
            prefetch_slot(WF, 8, a.z);
            break;
        case MG_OP_YCOL:
            prefetch_slot(WG, 4, a.z);
            prefetch_slot(WF, 8, a.w);
            break;
        case MG_OP_BIL:
        case MG_OP_AMP_SS:
            prefetch_slot(WF, 8, a.z);
            prefetch_slot(WF, 8, a.w);
            // the group sum it adds to (at L2) or reads
            if (a.x == MG_OP_AMP_SS && b.z >= 0 && !(b.w & 4)) prefetch_slot(ACC, 4, b.z);
            break;
        case MG_OP_AMP_VV:
            prefetch_slot(WG, 4, a.w);
            if (b.z >= 0 && !(b.w & 4)) prefetch_slot(ACC, 4, b.z);
            break;
        default:
            break;
    }
}

// The program of one item (same ops and semantics as the local-memory
// interpreter of mg_kernels.cu): pools G (slot s, component m: 4 s + m),
// F (slot s, variant v, component m: 8 s + 4 v + m), A (slot s, variant v:
// 4 s + v); jamp (c, v) of the item at jr[c * R / 2 + v * nipad] (real,
// imaginary).
// sde8 (may be NULL): per top-helicity combination v, |D_channel|^2 in [v]
// and the sum over the single-diagram-enhancement channels (the diagram
// terms of three-point vertices only) of |D|^2 in [4 + v].
template <int NG>
__device__ void run_item(const Kin<NG> &__restrict__ k, int g, const int4 *__restrict__ ops, int nops,
                         const int *__restrict__ scat, double mt, const Strided &WG,
                         const Strided &WF, const Strided &ACC, double2 *__restrict__ jr, long long R,
                         long long nipad, int channel, double *sde8) {
    cx G0[4][4];
    int4 an = __ldg(ops), bn = __ldg(ops + 1);
    for (int i = 0; i < nops; i++) {
        // this op's record was loaded one op ago; start the next record's
        // load and pull the next op's inputs towards L2 while this one runs
        const int4 a = an, b = bn;
        if (i + 1 < nops) {
            an = __ldg(ops + 2 * (i + 1));
            bn = __ldg(ops + 2 * (i + 1) + 1);
            prefetch_inputs(an, bn, WG, WF, ACC);
        }
        switch (a.x) {
            case MG_OP_EXT_G: {
                const int gi = (a.z < 2) ? a.z : a.z - 2;
                cx e[4];
                ext_gluon(k.P[a.z], ((g >> gi) & 1) ? 1 : -1, a.w != 0, e);
                WG.st4(4LL * a.y, e);
                break;
            }
            case MG_OP_EXT_UB:
            case MG_OP_EXT_V:
                for (int v = 0; v < 2; v++) {
                    cx o[4];
                    if (a.x == MG_OP_EXT_UB)
                        ext_ubar(k.P[2], v ? 1 : -1, o);
                    else
                        ext_v(k.P[3], v ? 1 : -1, o);
                    WF.st4(8LL * a.y + 4 * v, o);
                }
                break;
            case MG_OP_V3: {
                cx j1[4], j2[4], o[4];
                WG.ld4(4LL * a.z, j1);
                WG.ld4(4LL * a.w, j2);
                vvv_current(j1, k.K[b.x], j2, k.K[b.y], k.IP2[b.x | b.y], o);
                WG.st4(4LL * a.y, o);
                break;
            }
            case MG_OP_V4: {
                cx x[4], y[4], z[4], o1[4], o2[4], o3[4];
                WG.ld4(4LL * b.x, x);
                WG.ld4(4LL * b.y, y);
                WG.ld4(4LL * b.z, z);
                vvvv_currents(x, y, z, k.IP2[b.w], o1, o2, o3);
                WG.st4(4LL * a.y, o1);
                WG.st4(4LL * a.z, o2);
                WG.st4(4LL * a.w, o3);
                break;
            }
            case MG_OP_FPRE:
            case MG_OP_FSUF: {
                cx jg[4];
                WG.ld4(4LL * a.w, jg);
                const Slash s = slash_blocks(jg);
                const bool pre = a.x == MG_OP_FPRE;
                const cx d = pre ? k.DP[b.x] : k.DS[b.x];
                for (int v = 0; v < 2; v++) {
                    cx in[4], t[4], o[4];
                    WF.ld4(8LL * a.z + 4 * v, in);
                    if (pre) {
                        row_slash(in, s, t);
                        row_qm(t, k.QP[b.x], mt, o);
                    } else {
                        slash_col(s, in, t);
                        qm_col(k.QS[b.x], mt, t, o);
                    }
                    for (int m = 0; m < 4; m++) o[m] = o[m] * d;
                    WF.st4(8LL * a.y + 4 * v, o);
                }
                break;
            }
            case MG_OP_XROW:
            case MG_OP_YCOL: {
                const bool xrow = a.x == MG_OP_XROW;
                cx jg[4];
                WG.ld4(4LL * (xrow ? a.w : a.z), jg);
                const Slash s = slash_blocks(jg);
                for (int v = 0; v < 2; v++) {
                    cx in[4], o[4];
                    WF.ld4(8LL * (xrow ? a.z : a.w) + 4 * v, in);
                    if (xrow)
                        row_slash(in, s, o);
                    else
                        slash_col(s, in, o);
                    WF.st4(8LL * a.y + 4 * v, o);
                }
                break;
            }
            case MG_OP_BIL: {
                cx u[2][4], w[2][4];
                for (int v = 0; v < 2; v++) {
                    WF.ld4(8LL * a.z + 4 * v, u[v]);
                    WF.ld4(8LL * a.w + 4 * v, w[v]);
                }
                for (int bt = 0; bt < 2; bt++)
                    for (int btb = 0; btb < 2; btb++) bilinear(u[bt], w[btb], G0[2 * bt + btb]);
                break;
            }
            case MG_OP_AMP_SS:
            case MG_OP_AMP_VV: {
                cx amp[4];
                if (a.x == MG_OP_AMP_SS) {
                    cx x[2][4], y[2][4];
                    for (int v = 0; v < 2; v++) {
                        WF.ld4(8LL * a.z + 4 * v, x[v]);
                        WF.ld4(8LL * a.w + 4 * v, y[v]);
                    }
                    for (int bt = 0; bt < 2; bt++)
                        for (int btb = 0; btb < 2; btb++) amp[2 * bt + btb] = sdot(x[bt], y[btb]);
                } else {
                    cx w[4];
                    WG.ld4(4LL * a.w, w);
                    for (int v = 0; v < 4; v++) amp[v] = mdot(G0[v], w);
                }
                if (sde8 && a.y >= 0) {  // a diagram of three-point vertices: a channel
                    for (int v = 0; v < 4; v++) {
                        const double w = fma(amp[v].r, amp[v].r, amp[v].i * amp[v].i);
                        sde8[4 + v] += w;
                        if (a.y == channel) sde8[v] += w;
                    }
                }
                if (b.z >= 0) {  // member of a colour-factor group
                    // the group's sum: the first member stores, the middle
                    // ones add at L2, the last one reads it back (all
                    // relaxed: one thread's operations on an address stay in
                    // program order)
                    const int mode = b.w;
                    double2 *acc = ACC.p + 4LL * b.z * ACC.T;
                    if (!(mode & 8)) {
                        for (int v = 0; v < 4; v++) {
                            const cx t = unit_times(mode, amp[v]);
                            double2 *a = acc + v * ACC.T;
                            if (mode & 4)
                                st_relaxed(a, t);
                            else {
                                red_add(&a->x, t.r);
                                red_add(&a->y, t.i);
                            }
                        }
                        break;
                    }
                    for (int v = 0; v < 4; v++) {
                        const cx t = unit_times(mode, amp[v]);
                        amp[v] = (mode & 4) ? t : ld_relaxed(acc + v * ACC.T) + t;
                    }
                }
                // jamp updates as reductions at L2 (red.global.add.f64, no
                // value returned): the thread does not wait for the rows, and
                // the additions leave the FP64 pipe; a thread's reductions to
                // one address are applied in program order, so the sums are
                // the ones of a read-modify-write loop
                const int end = b.x + b.y;
                for (int s = b.x; s < end; s++) {
                    const int ev = __ldg(scat + s);
                    double2 *jc = jr + (long long)(ev >> 2) * (R / 2);
#pragma unroll
                    for (int v = 0; v < 4; v++) {
                        const cx t = unit_times(ev, amp[v]);
                        red_add(&jc[v * nipad].x, t.r);
                        red_add(&jc[v * nipad].y, t.i);
                    }
                }
                break;
            }
            default:
                break;
        }
    }
}

// The kinematic tables of every event of a chunk (Kin<7>: 17.7 KB), built
// once per event; every work item of the event reads them from there (the
// items of a warp share their event: broadcast loads, cached in L1) instead
// of building a copy in its own local memory.
template <int NG>
__global__ void k_kin_big(const double *__restrict__ mom, long long nevt, double mt, double wt,
                          Kin<NG> *__restrict__ kin) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nevt) kinematics<NG>(kin[e], mom + e * ((NG + 2) * 4), mt, wt);
}

// Four blocks per SM (128 registers, a few hundred bytes of spills): the
// 65,536 work items of 512 events then run as one wave of threads instead
// of two waves of half as many (measured 4.6% faster than three blocks).
template <int NG>
__global__ void __launch_bounds__(BIG_BLOCK, 4)
    k_sigmakin_big(const Kin<NG> *__restrict__ kin, long long nitem, int nunits,
                   const int *__restrict__ units, const int4 *__restrict__ ops, int nops,
                   const int *__restrict__ scat, double mt, double2 *__restrict__ scratch,
                   long long T, int nsg, int nsf, double *__restrict__ jrow, long long R,
                   long long nipad, int channel, const int *__restrict__ channel_ids,
                   double *__restrict__ sde_item) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const Strided WG{scratch + t, T};
    const Strided WF{scratch + 4LL * nsg * T + t, T};
    const Strided ACC{scratch + (4LL * nsg + 8LL * nsf) * T + t, T};
    for (long long item = t; item < nitem; item += T) {
        const long long e = item / nunits;
        const int u = __ldg(units + (item - e * nunits));
        double sde8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        run_item<NG>(kin[e], u >> 4, ops, nops, scat, mt, WG, WF, ACC,
                     reinterpret_cast<double2 *>(jrow) + item, R, nipad,
                     channel_ids ? __ldg(channel_ids + e) : channel, sde_item ? sde8 : nullptr);
        if (sde_item)
            for (int q = 0; q < 8; q++) sde_item[item * 8 + q] = sde8[q];
    }
}

// Colour sum of every row r over the block upper triangle:
// qpart[I * R + r] = sum_{n in tile I} V_rn Z_rn,  Z_rn = sum_{k >= 64 I} Cb_nk V_rk,
// with V_rk = jrow[k * R + r] and cbT[k * np + n] = Cb_nk.  Tile 64 rows x 64
// colours, 256 threads with 4 x 4 results each (thread (tx, ty): colours
// tx + 16 j, rows ty + 16 i), k in chunks of 16 through shared memory.
__global__ void __launch_bounds__(256)
    k_colour_big(const double *__restrict__ jrow, long long R, const double *__restrict__ cbT,
                 int np, double *__restrict__ qpart) {
    __shared__ double As[CK][RT];
    __shared__ double Bs[CK][CT];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long long r0 = (long long)blockIdx.x * RT;
    const int n0 = blockIdx.y * CT;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
    for (int k0 = n0; k0 < np; k0 += CK) {
#pragma unroll
        for (int q = 0; q < (CK * RT) / 256; q++) {
            const int idx = tid + 256 * q;
            const int kk = idx / RT, rr = idx % RT;
            As[kk][rr] = jrow[(long long)(k0 + kk) * R + r0 + rr];
            Bs[kk][rr] = cbT[(long long)(k0 + kk) * np + n0 + rr];
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < CK; kk++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const long long r = r0 + ty + 16 * i;
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < 4; j++) s = fma(jrow[(long long)(n0 + tx + 16 * j) * R + r], acc[i][j], s);
        for (int off = 8; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (tx == 0) qpart[(long long)blockIdx.y * R + r] = s;
    }
}

// Per event: sum over its items (units), good helicity combinations,
// real/imaginary rows and colour tiles, in that fixed order.
// Per-event extras: |M|^2 ~ alpha_s^NG, so alphas (may be NULL) rescales the
// event by (alphas[e] / alphas0)^NG; sde (with sde_item) is the event's
// channel weight over its good helicities.
template <int NG>
__global__ void k_event_sum_big(const double *__restrict__ qpart, long long R, int ntile,
                                long long nipad, const int *__restrict__ units, int nunits,
                                long long nevt, double factor, double *__restrict__ me,
                                double *__restrict__ me_hel, const double *__restrict__ alphas,
                                double alphas0, const double *__restrict__ sde_item,
                                double *__restrict__ sde) {
    constexpr int NPAR = NG + 2;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nevt) return;
    if (alphas) {
        const double r = alphas[e] / alphas0;
        for (int i = 0; i < NG; i++) factor *= r;
    }
    double num = 0.0, den = 0.0;
    double tot = 0.0;
    for (int iu = 0; iu < nunits; iu++) {
        const long long item = e * nunits + iu;
        const int u = __ldg(units + iu);
        for (int v = 0; v < 4; v++) {
            if (!((u >> v) & 1)) continue;
            double mh = 0.0;
            for (int ri = 0; ri < 2; ri++) {
                const long long r = 2 * (v * nipad + item) + ri;
                for (int I = 0; I < ntile; I++) mh += qpart[(long long)I * R + r];
            }
            tot += mh;
            if (me_hel) me_hel[e * (1LL << NPAR) + helicity_index<NG>(u >> 4, v >> 1, v & 1)] = mh * factor;
            if (sde_item) {
                num += sde_item[item * 8 + v];
                den += sde_item[item * 8 + 4 + v];
            }
        }
    }
    if (me) me[e] = tot * factor;
    if (sde) sde[e] = den > 0.0 ? num / den : 0.0;
}

// Helicity-summed |J_s|^2 per event and flow (jamps without couplings, good
// helicities only) from the FP64 jamp rows: jw[e * ncolor + c].
__global__ void k_flow_weights_big(const double *__restrict__ jrow, long long R, long long nipad,
                                   const int *__restrict__ units, int nunits, long long nevt,
                                   int ncolor, double *__restrict__ jw) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nevt * ncolor) return;
    const long long e = idx / ncolor;
    const int c = (int)(idx % ncolor);
    const double2 *col = reinterpret_cast<const double2 *>(jrow + (long long)c * R);
    double w = 0.0;
    for (int iu = 0; iu < nunits; iu++) {
        const long long item = e * nunits + iu;
        const int u = __ldg(units + iu);
        for (int v = 0; v < 4; v++) {
            if (!((u >> v) & 1)) continue;
            const double2 z = col[v * nipad + item];
            w = fma(z.x, z.x, fma(z.y, z.y, w));
        }
    }
    jw[idx] = w;
}

// Block upper triangle of D*C, transposed for the k-major tiles:
// cbT[k * np + n] = w * C_nk with w = 1 on the 64 x 64 diagonal blocks, 2
// above them, 0 below and in the padding.  C_nk = row[rank(r)] with r_i the
// position in ordering n of the i-th label of ordering k (the summed colour
// labels are dummies, so only the relative ordering matters).
template <int NG>
__global__ void k_build_cbig(const long long *__restrict__ row, const signed char *__restrict__ perm,
                             int nc, int np, double *__restrict__ cbT) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)np * np) return;
    const int k = (int)(idx / np), n = (int)(idx % np);
    const int bi = n / CT, bj = k / CT;
    double val = 0.0;
    if (n < nc && k < nc && bj >= bi) {
        int pos[NG];
        for (int a = 0; a < NG; a++) pos[perm[n * NG + a]] = a;
        long long rank = 0;
        unsigned used = 0;
        for (int i = 0; i < NG; i++) {
            const int ri = pos[perm[k * NG + i]];
            const int smaller = __popc(~used & ((1u << ri) - 1u));
            rank = rank * (NG - i) + smaller;
            used |= 1u << ri;
        }
        val = (double)row[rank] * (bj > bi ? 2.0 : 1.0);
    }
    cbT[idx] = val;
}

// Mixed precision: FP64 colour-major rows jrow[c * R + r] (c < nsrc) to the
// tensor-core rows jb[r * 3 kp + s * kp + c] (s = hi, mid, lo: the value
// rounded to FP32, then split twice into BF16), colours >= nsrc zero.
// Tiles of 64 rows x 64 colours through shared memory (reads coalesced along
// rows, writes along colours).
__global__ void __launch_bounds__(256)
    k_rows_to_bf16(const double *__restrict__ jrow, long long R, int nsrc, int kp,
                   __nv_bfloat16 *__restrict__ jb) {
    __shared__ double tile[64][65];
    const long long r0 = (long long)blockIdx.x * 64;
    const int c0 = blockIdx.y * 64;
    const int tid = threadIdx.x;
    for (int q = tid; q < 64 * 64; q += 256) {
        const int cc = q / 64, rr = q % 64;
        tile[cc][rr] = (c0 + cc < nsrc) ? jrow[(long long)(c0 + cc) * R + r0 + rr] : 0.0;
    }
    __syncthreads();
    for (int q = tid; q < 64 * 64; q += 256) {
        const int rr = q / 64, cc = q % 64;
        const float f = __double2float_rn(tile[cc][rr]);
        const __nv_bfloat16 hi = __float2bfloat16_rn(f);
        const float r1 = f - __bfloat162float(hi);
        const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
        const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
        __nv_bfloat16 *row = jb + (r0 + rr) * (long long)(3 * kp) + c0 + cc;
        row[0] = hi;
        row[kp] = mid;
        row[2 * kp] = lo;
    }
}

// D*C = C_hi + C_lo in BF16 for the tensor cores: cm[n * kp + k] = hi,
// cm[(kp + n) * kp + k] = lo, zero outside nc x nc.
template <int NG>
__global__ void k_build_cmat_bf16(const long long *__restrict__ row, const signed char *__restrict__ perm,
                                  int nc, int kp, __nv_bfloat16 *__restrict__ cm) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)kp * kp) return;
    const int n = (int)(idx / kp), k = (int)(idx % kp);
    float c = 0.0f;
    if (n < nc && k < nc) {
        int pos[NG];
        for (int a = 0; a < NG; a++) pos[perm[n * NG + a]] = a;
        long long rank = 0;
        unsigned used = 0;
        for (int i = 0; i < NG; i++) {
            const int ri = pos[perm[k * NG + i]];
            rank = rank * (NG - i) + __popc(~used & ((1u << ri) - 1u));
            used |= 1u << ri;
        }
        c = (float)row[rank];   // at most 15 significant bits: exact in FP32
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn(c);
    cm[idx] = hi;
    cm[(long long)kp * kp + idx] = __float2bfloat16_rn(c - __bfloat162float(hi));
}

}  // namespace

int mg_big_ngluon() { return BIG_NG; }

size_t mg_big_kin_bytes() { return sizeof(Kin<BIG_NG>); }

size_t mg_big_state_bytes(int nslot, int nslot_top, int nslot_acc) {
    return (size_t)(4LL * nslot + 8LL * nslot_top + 4LL * nslot_acc) * sizeof(double2);
}

int mg_big_block() { return BIG_BLOCK; }

int mg_big_blocks_per_sm(int *out) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_sigmakin_big<BIG_NG>, BIG_BLOCK, 0) ==
                   cudaSuccess
               ? 0
               : -1;
}

cudaError_t mg_launch_build_cbig(const long long *row, const signed char *perm, int nc, int np,
                                 double *cbT, cudaStream_t stream) {
    if (np % CT || np < nc) return cudaErrorInvalidValue;
    const long long n = (long long)np * np;
    mg_note_launch();
    k_build_cbig<BIG_NG><<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(row, perm, nc, np, cbT);
    return cudaGetLastError();
}

cudaError_t mg_launch_build_cmat_bf16(const long long *row, const signed char *perm, int nc, int kp,
                                     __nv_bfloat16 *cm, cudaStream_t stream) {
    if (kp < nc) return cudaErrorInvalidValue;
    const long long n = (long long)kp * kp;
    mg_note_launch();
    k_build_cmat_bf16<BIG_NG><<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(row, perm, nc, kp, cm);
    return cudaGetLastError();
}

cudaError_t mg_launch_rows_to_bf16(const double *jrow, long long R, int nsrc, int kp,
                                   __nv_bfloat16 *jb, cudaStream_t stream) {
    if (R <= 0) return cudaSuccess;
    if (R % 64 || kp % 64) return cudaErrorInvalidValue;
    mg_note_launch();
    k_rows_to_bf16<<<dim3((unsigned)(R / 64), (unsigned)(kp / 64)), 256, 0, stream>>>(jrow, R, nsrc, kp, jb);
    return cudaGetLastError();
}

cudaError_t mg_launch_sigmakin_big(const mg_dev_proc &dp, const double *mom, long long nitem,
                                   const int *units, int nunits, int nsg, int nsf, double2 *scratch,
                                   long long T, double *jrow, long long R, long long nipad,
                                   void *kin, cudaStream_t stream, int channel,
                                   const int *channel_ids, double *sde_item) {
    if (nitem <= 0) return cudaSuccess;
    if (T <= 0 || T % BIG_BLOCK || R != 8 * nipad || nipad < nitem || nunits <= 0 || !kin)
        return cudaErrorInvalidValue;
    const long long nevt = (nitem + nunits - 1) / nunits;
    Kin<BIG_NG> *k = static_cast<Kin<BIG_NG> *>(kin);
    mg_note_launch();
    k_kin_big<BIG_NG><<<(unsigned)((nevt + 63) / 64), 64, 0, stream>>>(mom, nevt, dp.mt, dp.wt, k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mg_note_launch();
    k_sigmakin_big<BIG_NG><<<(unsigned)(T / BIG_BLOCK), BIG_BLOCK, 0, stream>>>(
        k, nitem, nunits, units, reinterpret_cast<const int4 *>(dp.ops), dp.nops, dp.scat, dp.mt,
        scratch, T, nsg, nsf, jrow, R, nipad, channel, channel_ids, sde_item);
    return cudaGetLastError();
}

cudaError_t mg_launch_flow_weights_big(const double *jrow, long long R, long long nipad,
                                       const int *units, int nunits, long long nevt, int ncolor,
                                       double *jw, cudaStream_t stream) {
    if (nevt <= 0) return cudaSuccess;
    const long long n = nevt * ncolor;
    mg_note_launch();
    k_flow_weights_big<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(jrow, R, nipad, units, nunits,
                                                                         nevt, ncolor, jw);
    return cudaGetLastError();
}

cudaError_t mg_launch_colour_big(const double *jrow, long long R, const double *cbT, int np,
                                 double *qpart, cudaStream_t stream) {
    if (R <= 0) return cudaSuccess;
    if (R % RT || np % CT) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)(R / RT), (unsigned)(np / CT));
    mg_note_launch();
    k_colour_big<<<grid, 256, 0, stream>>>(jrow, R, cbT, np, qpart);
    return cudaGetLastError();
}

cudaError_t mg_launch_event_sum_big(const double *qpart, long long R, int ntile, long long nipad,
                                    const int *units, int nunits, long long nevt, double factor,
                                    double *me, double *me_hel, cudaStream_t stream,
                                    const double *alphas, double alphas0, const double *sde_item,
                                    double *sde) {
    if (nevt <= 0) return cudaSuccess;
    mg_note_launch();
    k_event_sum_big<BIG_NG><<<(unsigned)((nevt + 127) / 128), 128, 0, stream>>>(
        qpart, R, ntile, nipad, units, nunits, nevt, factor, me, me_hel, alphas, alphas0, sde_item,
        sde);
    return cudaGetLastError();
}
