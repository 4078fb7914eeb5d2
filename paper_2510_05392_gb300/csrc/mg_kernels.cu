// Diagram kernel: `tpe` threads per event share its work units (one
// gluon-helicity configuration with the four top/antitop helicities each),
// execute the process's wavefunction/amplitude program
// (compiler/program.py) and the FP64 colour sum, and the event's threads are
// reduced with warp shuffles.
//
// Structure of the paper's sigmaKin (Sec. 2.2): per event and good helicity,
// external wavefunctions -> internal wavefunctions -> amplitudes -> jamps ->
// quadratic form J^H C J (Sec. 3.3, Eq. "jcj", here sum_ij D*C_ij (A_i A_j +
// B_i B_j) with the symmetric matrix walked as an upper triangle, Sec. 3.3-3.4
// "triangular" colour sum) -> running sum over helicities.
//
// GB300 design notes.  The FP64 pipe is the bottleneck of this kernel by a
// wide margin, so the program is table driven: an op record is a uniform
// (warp-broadcast) load, the dispatch is warp-uniform, and wavefunctions,
// colour-group sums and per-event kinematics live in per-thread local memory.
// The jamps accumulate in a per-thread global buffer through FP64 reductions
// performed at L2 (red.global.add.f64: no wait for the old value, and the
// additions, about a tenth of the FP64 instructions, leave the FP64 pipe;
// measured +9% for ggttgg, +12% for ggttggg), then come back into local
// memory for the colour sum; without a buffer they stay in local memory and
// are updated in place.  Per-event
// quantities (momentum sums, 1/P^2, top propagators) are computed once per
// thread and reused by all of its helicities; gluon wavefunctions are shared
// by the four top/antitop helicities of a unit (helicity recycling of the
// FP64 work that does not depend on the top helicities).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mg_dirac.cuh"
#include "mg_internal.h"
#include "mg_kin.cuh"
#include "mg_proc_list.h"

using namespace mg;

namespace {

__device__ __forceinline__ void red_add(double *p, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed(double2 *p, double r, double i) {
    asm volatile("st.relaxed.gpu.global.v2.f64 [%0], {%1, %2};" ::"l"(p), "d"(r), "d"(i) : "memory");
}

__device__ __forceinline__ cx ld_relaxed(const double2 *p) {
    double r, i;
    asm volatile("ld.relaxed.gpu.global.v2.f64 {%0, %1}, [%2];" : "=d"(r), "=d"(i) : "l"(p) : "memory");
    return mk(r, i);
}

// One evaluation of the program: gluon-helicity configuration g and all four
// (top, antitop) helicity combinations v = 2*bt + btb at once.  Gluon
// wavefunctions (pool WG) are computed once for the four; top-line objects
// (pool WF) carry the two helicities of the top (ubar side) or of the antitop
// (v side); the bilinear G0, the amplitudes and the jamps carry all four.
// Writes me4[v] = sum_ij D*C_ij Re(J_v,i^* J_v,j).  With sde8, adds per
// variant v the |D|^2 of the single-diagram-enhancement channel `channel` to
// sde8[v] and of every channel to sde8[4 + v] (a channel's amplitude is the
// value of its one diagram term; its colour coefficients have modulus one).
// With jt (this thread's jamp buffer in global memory, jamp (c, v) at
// jt[(4 c + v) * js]) the jamp updates are FP64 reductions performed at L2
// (red.global.add.f64): the thread does not wait for them and the additions
// leave the FP64 pipe; the finished jamps are then read back into J.  A
// thread's zeroing stores, reductions and loads of one address are all
// relaxed (strong) operations, so they take effect in program order and the
// sums are the ones of the read-modify-write loop.
template <int NG, int NSG, int NSF, int NSA, int NC>
__device__ void run_unit(const Kin<NG> &k, int g, const int4 *__restrict__ ops, int nops,
                         const int *__restrict__ scat, const double *__restrict__ cup, double mt,
                         cx (*WG)[4], cx (*WF)[2][4], cx (*G0)[4], cx (*ACC)[4], cx (*J)[4],
                         double *me4, bool colour_sum, int channel = -1, double *sde8 = nullptr,
                         double2 *jt = nullptr, long long js = 0) {
    if (jt) {
        for (int i = 0; i < 4 * NC; i++) st_relaxed(jt + i * js, 0.0, 0.0);
    } else {
        for (int c = 0; c < NC; c++)
            for (int v = 0; v < 4; v++) J[c][v] = mk(0.0, 0.0);
    }
    for (int i = 0; i < nops; i++) {
        const int4 a = __ldg(ops + 2 * i);
        const int4 b = __ldg(ops + 2 * i + 1);
        switch (a.x) {
            case MG_OP_EXT_G: {
                const int gi = (a.z < 2) ? a.z : a.z - 2;
                ext_gluon(k.P[a.z], ((g >> gi) & 1) ? 1 : -1, a.w != 0, WG[a.y]);
                break;
            }
            case MG_OP_EXT_UB:
                ext_ubar(k.P[2], -1, WF[a.y][0]);
                ext_ubar(k.P[2], 1, WF[a.y][1]);
                break;
            case MG_OP_EXT_V:
                ext_v(k.P[3], -1, WF[a.y][0]);
                ext_v(k.P[3], 1, WF[a.y][1]);
                break;
            case MG_OP_V3:
                vvv_current(WG[a.z], k.K[b.x], WG[a.w], k.K[b.y], k.IP2[b.x | b.y], WG[a.y]);
                break;
            case MG_OP_V4:
                vvvv_currents(WG[b.x], WG[b.y], WG[b.z], k.IP2[b.w], WG[a.y], WG[a.z], WG[a.w]);
                break;
            case MG_OP_FPRE: {
                const Slash s = slash_blocks(WG[a.w]);
                const cx d = k.DP[b.x];
                for (int v = 0; v < 2; v++) {
                    cx t[4], o[4];
                    row_slash(WF[a.z][v], s, t);
                    row_qm(t, k.QP[b.x], mt, o);
                    for (int m = 0; m < 4; m++) WF[a.y][v][m] = o[m] * d;
                }
                break;
            }
            case MG_OP_FSUF: {
                const Slash s = slash_blocks(WG[a.w]);
                const cx d = k.DS[b.x];
                for (int v = 0; v < 2; v++) {
                    cx t[4], o[4];
                    slash_col(s, WF[a.z][v], t);
                    qm_col(k.QS[b.x], mt, t, o);
                    for (int m = 0; m < 4; m++) WF[a.y][v][m] = o[m] * d;
                }
                break;
            }
            case MG_OP_XROW: {
                const Slash s = slash_blocks(WG[a.w]);
                for (int v = 0; v < 2; v++) row_slash(WF[a.z][v], s, WF[a.y][v]);
                break;
            }
            case MG_OP_YCOL: {
                const Slash s = slash_blocks(WG[a.z]);
                for (int v = 0; v < 2; v++) slash_col(s, WF[a.w][v], WF[a.y][v]);
                break;
            }
            case MG_OP_BIL:
                for (int bt = 0; bt < 2; bt++)
                    for (int btb = 0; btb < 2; btb++) bilinear(WF[a.z][bt], WF[a.w][btb], G0[2 * bt + btb]);
                break;
            case MG_OP_AMP_SS:
            case MG_OP_AMP_VV: {
                cx amp[4];
                if (a.x == MG_OP_AMP_SS) {
                    for (int bt = 0; bt < 2; bt++)
                        for (int btb = 0; btb < 2; btb++)
                            amp[2 * bt + btb] = sdot(WF[a.z][bt], WF[a.w][btb]);
                } else {
                    for (int v = 0; v < 4; v++) amp[v] = mdot(G0[v], WG[a.w]);
                }
                if (sde8 && a.y >= 0) {  // a diagram of three-point vertices: a channel
                    for (int v = 0; v < 4; v++) {
                        const double w = fma(amp[v].r, amp[v].r, amp[v].i * amp[v].i);
                        sde8[4 + v] += w;
                        if (a.y == channel) sde8[v] += w;
                    }
                }
                if (b.z >= 0) {  // member of a colour-factor group
                    const int mode = b.w;
                    if (mode & 4) {
                        for (int v = 0; v < 4; v++) ACC[b.z][v] = unit_times(mode, amp[v]);
                    } else {
                        for (int v = 0; v < 4; v++) ACC[b.z][v] = ACC[b.z][v] + unit_times(mode, amp[v]);
                    }
                    if (!(mode & 8)) break;
                    for (int v = 0; v < 4; v++) amp[v] = ACC[b.z][v];
                }
                const int end = b.x + b.y;
                if (jt) {
                    for (int s = b.x; s < end; s++) {
                        const int e = __ldg(scat + s);
                        double2 *jc = jt + (long long)(4 * (e >> 2)) * js;
#pragma unroll
                        for (int v = 0; v < 4; v++) {
                            const cx t = unit_times(e, amp[v]);
                            red_add(&jc[v * js].x, t.r);
                            red_add(&jc[v * js].y, t.i);
                        }
                    }
                    break;
                }
                // jamp updates in pairs: the flows of one scatter list are
                // distinct, so both old values are loaded before either store
                // and the two loads wait for memory together
                int s = b.x;
                for (; s + 1 < end; s += 2) {
                    const int e0 = __ldg(scat + s), e1 = __ldg(scat + s + 1);
                    cx o0[4], o1[4];
#pragma unroll
                    for (int v = 0; v < 4; v++) {
                        o0[v] = J[e0 >> 2][v];
                        o1[v] = J[e1 >> 2][v];
                    }
#pragma unroll
                    for (int v = 0; v < 4; v++) {
                        J[e0 >> 2][v] = o0[v] + unit_times(e0, amp[v]);
                        J[e1 >> 2][v] = o1[v] + unit_times(e1, amp[v]);
                    }
                }
                if (s < end) {
                    const int e = __ldg(scat + s);
#pragma unroll
                    for (int v = 0; v < 4; v++) J[e >> 2][v] = J[e >> 2][v] + unit_times(e, amp[v]);
                }
                break;
            }
            default:
                break;
        }
    }
    if (jt)
        for (int c = 0; c < NC; c++)
            for (int v = 0; v < 4; v++) J[c][v] = ld_relaxed(jt + (4LL * c + v) * js);
    if (!colour_sum) return;
    // colour sum over the packed upper triangle (diagonal D*C_ii, off-diagonal
    // 2*D*C_ij), the four helicity combinations sharing each matrix entry
    double me[4] = {0.0, 0.0, 0.0, 0.0};
    const double *c = cup;
    for (int i = 0; i < NC; i++) {
        double zr[4] = {0.0, 0.0, 0.0, 0.0}, zi[4] = {0.0, 0.0, 0.0, 0.0};
        for (int j = i; j < NC; j++) {
            const double cij = __ldg(c++);
#pragma unroll
            for (int v = 0; v < 4; v++) {
                zr[v] = fma(cij, J[j][v].r, zr[v]);
                zi[v] = fma(cij, J[j][v].i, zi[v]);
            }
        }
#pragma unroll
        for (int v = 0; v < 4; v++) me[v] = fma(J[i][v].r, zr[v], fma(J[i][v].i, zi[v], me[v]));
    }
    for (int v = 0; v < 4; v++) me4[v] = me[v];
}

// Jamps of one unit as GEMM rows for the tensor-core colour sum: row
// m = ((e * nunits_pad + iu) * 4 + v) * 2 + (0: real, 1: imaginary part),
// each [3][kp] BF16 pieces hi, mid, lo with x ~= hi + mid + lo (the FP64 value
// rounded to FP32, then split twice); colours >= NC and masked-out helicity
// combinations are written as zeros.
template <int NC>
__device__ void write_jamp_rows(const cx (*J)[4], int mask, __nv_bfloat16 *__restrict__ jout,
                                long long row0, int kp) {
    for (int v = 0; v < 4; v++) {
        const bool on = (mask >> v) & 1;
        for (int ri = 0; ri < 2; ri++) {
            __nv_bfloat16 *row = jout + (row0 + 2 * v + ri) * (long long)(3 * kp);
            for (int c0 = 0; c0 < kp; c0 += 8) {
                if (!on || c0 >= NC) {  // padding colours, masked-out helicities: zeros
                    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
                    *reinterpret_cast<uint4 *>(row + c0) = z;
                    *reinterpret_cast<uint4 *>(row + kp + c0) = z;
                    *reinterpret_cast<uint4 *>(row + 2 * kp + c0) = z;
                    continue;
                }
                // only real colours pay for the FP64 -> FP32 conversion (an
                // FP64-pipe instruction); the BF16 splitting runs in FP32
                __align__(16) __nv_bfloat16 hi[8], mid[8], lo[8];
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int c = c0 + q;
                    float f = 0.0f;
                    if (c < NC) f = __double2float_rn(ri ? J[c][v].i : J[c][v].r);
                    hi[q] = __float2bfloat16_rn(f);
                    const float r1 = f - __bfloat162float(hi[q]);
                    mid[q] = __float2bfloat16_rn(r1);
                    lo[q] = __float2bfloat16_rn(r1 - __bfloat162float(mid[q]));
                }
                *reinterpret_cast<uint4 *>(row + c0) = *reinterpret_cast<const uint4 *>(hi);
                *reinterpret_cast<uint4 *>(row + kp + c0) = *reinterpret_cast<const uint4 *>(mid);
                *reinterpret_cast<uint4 *>(row + 2 * kp + c0) = *reinterpret_cast<const uint4 *>(lo);
            }
        }
    }
}

// Plain instantiations: three 128-thread blocks per SM (167 registers, no
// spills; the FP64 pipe then has 12 warps to hide local-memory latency with);
// the extras instantiation keeps the register budget of 256-thread blocks.
template <int NG, int NSG, int NSF, int NSA, int NC, bool EX>
__global__ void __launch_bounds__(EX ? 256 : 128, EX ? 1 : 3)
    k_sigmakin(const double *__restrict__ mom, long long nevt, const int4 *__restrict__ ops,
               int nops, const int *__restrict__ scat, const double *__restrict__ cup,
               const int *__restrict__ units, int nunits, int tpe, double mt, double wt,
               double factor, double *__restrict__ me, double *__restrict__ me_hel,
               __nv_bfloat16 *__restrict__ jout, int kp, int nunits_pad, mg_extras ex,
               double2 *__restrict__ jg) {
    constexpr int NPAR = NG + 2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long js = (long long)gridDim.x * blockDim.x;   // jamp buffer stride
    const long long e = t / tpe;
    const int s = (int)(t - e * tpe);
    double sum = 0.0;
    // per-event extras (compiled only into the EX instantiation)
    double sde8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int channel = (EX && ex.channel_ids && e < nevt) ? __ldg(ex.channel_ids + e) : ex.channel;
    double num = 0.0, den = 0.0;
    double jw[EX ? NC : 1];
    if (EX && ex.jw)
        for (int c = 0; c < NC; c++) jw[c] = 0.0;
    if (EX && ex.alphas && e < nevt) {  // per-event strong coupling: |M|^2 ~ alpha_s^NG
        const double r = ex.alphas[e] / ex.alphas0;
        double f = 1.0;
        for (int i = 0; i < NG; i++) f *= r;
        factor *= f;
    }
    if (e < nevt) {
        Kin<NG> k;
        kinematics<NG>(k, mom + e * (NPAR * 4), mt, wt);
        cx WG[NSG > 0 ? NSG : 1][4];
        cx WF[NSF > 0 ? NSF : 1][2][4];
        cx G0[4][4];
        cx ACC[NSA][4];
        cx J[NC][4];
        for (int iu = s; iu < nunits; iu += tpe) {
            const int u = __ldg(units + iu);
            const int g = u >> 4, mask = u & 15;
            double me4[4];
            if (EX)
                for (int q = 0; q < 8; q++) sde8[q] = 0.0;
            run_unit<NG, NSG, NSF, NSA, NC>(k, g, ops, nops, scat, cup, mt, WG, WF, G0, ACC, J, me4,
                                            !jout, channel, (EX && ex.sde) ? sde8 : nullptr,
                                            jg ? jg + t : nullptr, js);
            if (jout) {
                write_jamp_rows<NC>(J, mask, jout, (e * nunits_pad + iu) * 8, kp);
                continue;
            }
            for (int v = 0; v < 4; v++) {
                if (!((mask >> v) & 1)) continue;
                sum += me4[v];
                if (EX) {
                    num += sde8[v];
                    den += sde8[4 + v];
                    if (ex.jw)
                        for (int c = 0; c < NC; c++)
                            jw[c] = fma(J[c][v].r, J[c][v].r, fma(J[c][v].i, J[c][v].i, jw[c]));
                }
                if (me_hel) me_hel[e * (1LL << NPAR) + helicity_index<NG>(g, v >> 1, v & 1)] = me4[v] * factor;
            }
        }
    }
    for (int o = tpe >> 1; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (EX && ex.sde) {
            num += __shfl_xor_sync(0xffffffffu, num, o);
            den += __shfl_xor_sync(0xffffffffu, den, o);
        }
        if (EX && ex.jw)
            for (int c = 0; c < NC; c++) jw[c] += __shfl_xor_sync(0xffffffffu, jw[c], o);
    }
    if (e < nevt && s == 0) {
        if (me) me[e] = sum * factor;
        if (EX && ex.sde) ex.sde[e] = den > 0.0 ? num / den : 0.0;
        if (EX && ex.jw)
            for (int c = 0; c < NC; c++) ex.jw[e * NC + c] = jw[c];
    }
}

// Helicity and colour-flow choice per event (the other output of the
// paper's sigmaKin, Sec. 2.2): h is the first index whose running sum of
// |M_h|^2 exceeds r_hel times the total, the flow likewise from the
// helicity-summed |J_s|^2.
__global__ void k_select(const double *__restrict__ me_hel, int nhel, const double *__restrict__ jw,
                         int ncolor, long long nevt, const double *__restrict__ rh,
                         const double *__restrict__ rc, int *__restrict__ hel_out,
                         int *__restrict__ col_out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nevt) return;
    if (hel_out && rh) {
        const double *w = me_hel + e * nhel;
        double tot = 0.0;
        for (int h = 0; h < nhel; h++) tot += w[h];
        const double cut = rh[e] * tot;
        double run = 0.0;
        int pick = -1;
        for (int h = 0; h < nhel; h++) {
            if (w[h] <= 0.0) continue;
            run += w[h];
            pick = h;
            if (run > cut) break;
        }
        hel_out[e] = pick;
    }
    if (col_out && rc) {
        const double *w = jw + e * ncolor;
        double tot = 0.0;
        for (int c = 0; c < ncolor; c++) tot += w[c];
        const double cut = rc[e] * tot;
        double run = 0.0;
        int pick = -1;
        for (int c = 0; c < ncolor; c++) {
            if (w[c] <= 0.0) continue;
            run += w[c];
            pick = c;
            if (run > cut) break;
        }
        col_out[e] = pick;
    }
}

// ------------------------------------------------ multi-process batch ----
// One slot of a batch item: event e = slot / tpe, thread s = slot % tpe of that
// event.  All 32 lanes of a warp call this for the same item (the shuffles
// below span the warp).  Kept out of line so that the persistent kernel's
// stack frame is the largest of the carried processes, not their sum.
// jt: this thread's jamp buffer (stride js), or NULL.
template <int NG, int NSG, int NSF, int NSA, int NC>
__device__ __noinline__ void batch_slot(const mg_batch_item &it, long long slot, double2 *jt,
                                        long long js) {
    constexpr int NPAR = NG + 2;
    const int tpe = it.tpe;
    const long long e = slot / tpe;
    const int s = (int)(slot - e * tpe);
    double sum = 0.0;
    if (e < it.nevt) {
        Kin<NG> k;
        kinematics<NG>(k, it.mom + e * (NPAR * 4), it.mt, it.wt);
        cx WG[NSG > 0 ? NSG : 1][4];
        cx WF[NSF > 0 ? NSF : 1][2][4];
        cx G0[4][4];
        cx ACC[NSA][4];
        cx J[NC][4];
        const int4 *ops = reinterpret_cast<const int4 *>(it.ops);
        for (int iu = s; iu < it.nunits; iu += tpe) {
            const int u = __ldg(it.units + iu);
            double me4[4];
            run_unit<NG, NSG, NSF, NSA, NC>(k, u >> 4, ops, it.nops, it.scat, it.cup, it.mt, WG, WF,
                                            G0, ACC, J, me4, true, -1, nullptr, jt, js);
            for (int v = 0; v < 4; v++)
                if ((u >> v) & 1) sum += me4[v];
        }
    }
    for (int o = tpe >> 1; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (e < it.nevt && s == 0) it.me[e] = sum * it.factor;
}

template <int NG, int NSG, int NSF, int NSA, int NC>
__device__ __forceinline__ void batch_dispatch(const mg_batch_item &it, long long slot, double2 *jt,
                                               long long js) {
    if constexpr (NG <= MG_BATCH_MAX_NGLUON) batch_slot<NG, NSG, NSF, NSA, NC>(it, slot, jt, js);
}

// Persistent kernel: every warp repeatedly takes the next 32 slots from the
// global counter until all items are done (no waits on other threads).
// jg (may be NULL): jamp buffers, thread t's jamp (c, v) at
// jg[(4 c + v) * T + t], T = the launch's threads.
__global__ void __launch_bounds__(128, 3)
    k_batch(const mg_batch_item *__restrict__ items, int nitems,
            unsigned long long *__restrict__ counter, long long total_slots, double2 *__restrict__ jg) {
    const int lane = threadIdx.x & 31;
    const long long js = (long long)gridDim.x * blockDim.x;
    double2 *jt = jg ? jg + (long long)blockIdx.x * blockDim.x + threadIdx.x : nullptr;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(counter, 32ULL);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((long long)base >= total_slots) return;
        int i = 0;
        while (i + 1 < nitems && (long long)base >= items[i].slot_end) i++;
        const mg_batch_item &it = items[i];
        const long long slot = (long long)base + lane - it.slot_begin;
        switch (it.table_index) {
#define MG_BATCH_CASE(IDX, NG, NSG, NSF, NSA, NC) \
    case IDX:                                     \
        batch_dispatch<NG, NSG, NSF, NSA, NC>(it, slot, jt, js); \
        break;
            MG_PROC_LIST(MG_BATCH_CASE)
#undef MG_BATCH_CASE
            default:
                break;
        }
    }
}

// Helicity filter rule: good[h] = any_e ( mh[e][h] > rel * max_h' mh[e][h'] ).
__global__ void k_helmask(const double *__restrict__ mh, long long n, int nhel, double rel,
                          unsigned char *__restrict__ mask) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= nhel) return;
    unsigned char good = 0;
    for (long long e = 0; e < n; e++) {
        const double *row = mh + e * nhel;
        double mx = 0.0;
        for (int j = 0; j < nhel; j++) mx = fmax(mx, row[j]);
        if (row[h] > rel * mx) good = 1;
    }
    mask[h] = good;
}

}  // namespace

cudaError_t mg_launch_sigmakin(const mg_dev_proc &dp, const double *mom, int64_t nevt,
                               const int *units, int nunits, int tpe, int block, double *me,
                               double *me_hel, cudaStream_t stream, __nv_bfloat16 *jout, int kp,
                               int nunits_pad, const mg_extras *extras, double2 *jg) {
    mg_extras ex;
    if (extras) {
        ex = *extras;
    } else {
        ex.alphas = nullptr;
        ex.alphas0 = 1.0;
        ex.channel = -1;
        ex.channel_ids = nullptr;
        ex.sde = nullptr;
        ex.jw = nullptr;
    }
    if (nevt <= 0) return cudaSuccess;
    const long long threads = (long long)nevt * tpe;
    const long long grid = (threads + block - 1) / block;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
    mg_note_launch();
    switch (dp.table_index) {
#define MG_LAUNCH(IDX, NG, NSG, NSF, NSA, NC)                                                    \
    case IDX:                                                                                    \
        if (extras)                                                                              \
            k_sigmakin<NG, NSG, NSF, NSA, NC, true><<<(unsigned)grid, block, 0, stream>>>(       \
                mom, nevt, reinterpret_cast<const int4 *>(dp.ops), dp.nops, dp.scat, dp.cup,      \
                units, nunits, tpe, dp.mt, dp.wt, dp.factor, me, me_hel, jout, kp, nunits_pad, ex, jg); \
        else                                                                                     \
            k_sigmakin<NG, NSG, NSF, NSA, NC, false><<<(unsigned)grid, block, 0, stream>>>(      \
                mom, nevt, reinterpret_cast<const int4 *>(dp.ops), dp.nops, dp.scat, dp.cup,      \
                units, nunits, tpe, dp.mt, dp.wt, dp.factor, me, me_hel, jout, kp, nunits_pad, ex, jg); \
        break;
        MG_PROC_LIST(MG_LAUNCH)
#undef MG_LAUNCH
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t mg_launch_helmask(const double *me_hel, int64_t n, int nhel, double rel,
                              unsigned char *mask, cudaStream_t stream) {
    mg_note_launch();
    k_helmask<<<(nhel + 127) / 128, 128, 0, stream>>>(me_hel, n, nhel, rel, mask);
    return cudaGetLastError();
}

cudaError_t mg_launch_batch(const mg_batch_item *d_items, int nitems, unsigned long long *d_counter,
                            long long total_slots, int grid, cudaStream_t stream, double2 *jg) {
    cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    if (total_slots <= 0) return cudaSuccess;
    mg_note_launch();
    k_batch<<<grid, 128, 0, stream>>>(d_items, nitems, d_counter, total_slots, jg);
    return cudaGetLastError();
}

int mg_batch_ctas_per_sm(int *out) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch, 128, 0) != cudaSuccess)
        return MG_ERR_CUDA;
    *out = n;
    return MG_OK;
}

// CTAs of the process's diagram kernel resident per SM at this block size.
int mg_sigmakin_occupancy(int table_index, int block, int *ctas_per_sm) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (table_index) {
#define MG_OCC(IDX, NG, NSG, NSF, NSA, NC)                                                       \
    case IDX:                                                                                    \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sigmakin<NG, NSG, NSF, NSA, NC, false>, \
                                                          block, 0);                             \
        break;
        MG_PROC_LIST(MG_OCC)
#undef MG_OCC
        default:
            break;
    }
    if (e != cudaSuccess) return MG_ERR_CUDA;
    *ctas_per_sm = n > 0 ? n : 1;
    return MG_OK;
}

cudaError_t mg_launch_select(const double *me_hel, int nhel, const double *jw, int ncolor,
                             long long nevt, const double *rh, const double *rc, int *hel_out,
                             int *col_out, cudaStream_t stream) {
    if (nevt <= 0) return cudaSuccess;
    mg_note_launch();
    k_select<<<(unsigned)((nevt + 127) / 128), 128, 0, stream>>>(me_hel, nhel, jw, ncolor, nevt, rh, rc,
                                                               hel_out, col_out);
    return cudaGetLastError();
}
