// Colour sum on the tensor cores (tcgen05, sm_103a): the mixed-precision
// variant of the paper's colour sum J^H C J = A^T C A + B^T C B (Sec. 3.3,
// Eq. "jcj"; Sec. 3.4 runs it as one GEMM over all helicities).
//
// Columns.  Every real vector V (the real or the imaginary part of the jamps
// of one event and helicity) is a GEMM row m of length ncolor, stored as
// three BF16 pieces V = V_hi + V_mid + V_lo (about 24 significant bits), each
// padded to KP colours:  jbuf[m][s*KP + c], s = hi, mid, lo.
// The colour matrix D*C (integers, not all exact in BF16 for 120 flows) is
// split C_hat = C_hi + C_lo, both exact in BF16:  cmat[h*NP + n][c].
//
// One CTA computes Z = V C_hat^T for 128 columns (M = 128, N = NP colours,
// K = KP per piece) with FP32 accumulation in tensor memory:
//   Z = sum_{s in hi,mid,lo} V_s C_hi  +  sum_{s in hi,mid} V_s C_lo
// (V_lo C_lo, relatively ~2^-24, is dropped), then the epilogue threads read
// Z from TMEM and form sum_n V[m][n] Z[m][n] (compensated FP32, V = hi + mid
// + lo from the operand tiles already in shared memory).  Partial sums go to
// part[] in a fixed layout; k_event_sum adds each event's partials in order.
//
// Operands reach shared memory by TMA (cp.async.bulk.tensor, 128-byte
// swizzle, box 64 x rows); one elected thread issues tcgen05.mma and
// tcgen05.commit; every wait on an mbarrier is bounded (about a second): on
// timeout the warp records MG_TC_ERR_TIMEOUT in *err and a CTA-wide flag that
// stops the other roles at their next wait, and the CTA frees its tensor
// memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mg_internal.h"
#include "mg_tc.cuh"

namespace {

using namespace mgtc;

// Warp-specialised persistent kernel (2 + 8 TC_NSPLIT warps):
//   warp 0  TMA producer: the two colour-matrix halves once, then the A chunks
//           (one split x KW colours x 128 rows: 16 KiB at KW = 64, 8 KiB at
//           KW = 32 for up to 32 flows) of every tile through
//           a ring of TC_STAGES shared-memory stages (full/empty mbarriers);
//   warp 1  MMA issuer (one thread): per chunk KW / 16 (hi) or KW / 8 (hi +
//           lo colour matrix) tcgen05.mma, then tcgen05.commit to the stage's "empty"
//           barrier; per tile a commit to the accumulator's "full" barrier;
//           two TMEM accumulators alternate between the CTA's tiles;
//   warps 2.. epilogue, two groups: group a takes the CTA's tiles i with
//           i % 2 = a and TMEM accumulator a, so one group reads the next
//           tile's operands (and frees their stages) while the other forms
//           its sums.  In a group each thread owns one row (TMEM lane
//           32 (warp % 4) + lane) and one of TC_NSPLIT colour sets, the
//           16-colour groups g with g % TC_NSPLIT equal to its set.  A thread
//           reads its row's colours from every A chunk in the stage the MMAs
//           read (128-byte swizzle: 16-byte piece j of row m sits at piece
//           j ^ (m % 8); 64-byte swizzle: at j ^ ((m / 2) % 4); a warp's
//           reads are conflict-free either way) and sums
//           V = hi + mid + lo in registers; a stage is free once the MMA
//           commit and the 4 TC_NSPLIT warps of the tile's group have
//           arrived.  After the accumulator lands the thread forms its part of
//           sum_n V Z in compensated FP32 (exact products, two-sum
//           accumulation, ~48 significant bits), sums it in FP64 over the
//           lanes of its event group (butterfly, fixed order) and writes one
//           partial per warp segment to part[]; no two epilogue warps wait
//           for each other.
// The jamp rows are read from HBM exactly once (by TMA).
constexpr int TC_STAGES = 8;   // deeper rings (10, 12) measured no faster
constexpr int TC_NSPLIT = 2;                  // colour sets per row
constexpr int TC_NGROUP = 2;                  // epilogue groups, one per TMEM accumulator
constexpr int TC_GROUP_WARPS = 4 * TC_NSPLIT;
constexpr int TC_EPI_WARPS = TC_NGROUP * TC_GROUP_WARPS;
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;
// Each epilogue group has a ring of its own (stages [TC_RING g, TC_RING (g + 1))):
// a stage is then filled and released by one group only, in order, so a
// parity wait can never mistake another group's earlier fill for its own.
constexpr int TC_RING = TC_STAGES / TC_NGROUP;

__device__ __forceinline__ void ring_slot(int grp, long long q, int &stage, uint32_t &phase) {
    stage = grp * TC_RING + (int)(q % TC_RING);
    phase = (uint32_t)((q / TC_RING) & 1);
}

struct TcSmem {
    uint64_t *bB, *full, *empty, *tfull, *tempty;
    uint32_t *tmem_slot;
    int *failed;
};

__device__ __forceinline__ void tc_fail(int *failed, int *err) {
    atomicExch(failed, 1);
    atomicExch(err, MG_TC_ERR_TIMEOUT);
}

// KW colours per chunk (64: 128-byte rows and swizzle; 32: 64-byte rows and
// swizzle, for up to 32 flows, so 24 flows read 1.33x their bytes instead of
// 2.67x); KCN = kp / KW colour chunks per split (1 for up to KW colours, 2 for
// up to 128).
template <int KW, int KCN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_colorsum_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  int np, int np_pad, int cpe, long long ntiles, int tmem_cols, uint32_t extra_tx,
                  double *__restrict__ part, int *__restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int kc_n = KCN;
    constexpr int kp = KCN * KW;
    constexpr int nchunk = 3 * KCN;             // A chunks per tile: split-major
    constexpr int RB = 2 * KW;                  // bytes per row of a chunk
    constexpr int GPC = KW / 16;                // 16-colour groups per chunk
    static_assert((KW == 32 || KW == TC_KCHUNK) && GPC % TC_NSPLIT == 0, "chunk width");
    const int a_chunk = TC_M * RB;
    const int b_chunk = np * RB;
    unsigned char *sB = smem;                   // [2][kc_n] chunks, resident
    unsigned char *sA = sB + 2 * kc_n * b_chunk;  // [TC_STAGES] chunks
    uint64_t *bars = reinterpret_cast<uint64_t *>(sA + TC_STAGES * a_chunk);
    TcSmem S;
    S.bB = bars;
    S.full = bars + 1;
    S.empty = S.full + TC_STAGES;
    S.tfull = S.empty + TC_STAGES;
    S.tempty = S.tfull + 2;
    S.tmem_slot = reinterpret_cast<uint32_t *>(S.tempty + 2);
    S.failed = reinterpret_cast<int *>(S.tmem_slot + 1);


    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(S.tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        mbar_init(S.bB, 1);
        for (int i = 0; i < TC_STAGES; i++) {
            mbar_init(&S.full[i], 1);
            mbar_init(&S.empty[i], 1 + TC_GROUP_WARPS);   // MMA commit + the tile's epilogue group
        }
        for (int i = 0; i < 2; i++) {
            mbar_init(&S.tfull[i], 1);
            mbar_init(&S.tempty[i], TC_GROUP_WARPS);   // one arrival per warp of the group
        }
        *S.failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *S.tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // ------------------------------------ producer
            mbar_expect_tx(S.bB, (uint32_t)(2 * kc_n * b_chunk));
            for (int h = 0; h < 2; h++)
                for (int kc = 0; kc < kc_n; kc++)
                    tma_load_2d(sB + (h * kc_n + kc) * b_chunk, &tmB, kc * KW, h * np, S.bB);
            long long q[TC_NGROUP] = {0, 0};   // fills per ring
            int k = 0;                          // tile index among this CTA's tiles
            for (long long t = blockIdx.x; t < ntiles && !*(volatile int *)S.failed; t += gridDim.x, k++) {
                const int g = k % TC_NGROUP;
                for (int c = 0; c < nchunk; c++) {
                    int stage;
                    uint32_t phase;
                    ring_slot(g, q[g]++, stage, phase);
                    if (!mbar_wait(&S.empty[stage], phase ^ 1, TC_WAIT_CYCLES)) {
                        tc_fail(S.failed, err);
                        break;
                    }
                    mbar_expect_tx(&S.full[stage], (uint32_t)a_chunk + extra_tx);
                    const int sp = c / kc_n, kc = c % kc_n;
                    tma_load_2d(sA + stage * a_chunk, &tmA, sp * kp + kc * KW, (int)(t * TC_M),
                                &S.full[stage]);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ------------------------------------ MMA issuer
            bool ok = mbar_wait(S.bB, 0, TC_WAIT_CYCLES);
            if (!ok) tc_fail(S.failed, err);
            const uint32_t idesc = instr_desc(TC_M, np);
            long long q[TC_NGROUP] = {0, 0};   // fills per ring
            uint32_t aphase = 0;
            int acc = 0;                        // = tile index % 2 = the tile's group
            for (long long t = blockIdx.x; ok && t < ntiles && !*(volatile int *)S.failed; t += gridDim.x) {
                if (!mbar_wait(&S.tempty[acc], aphase ^ 1, TC_WAIT_CYCLES)) {
                    tc_fail(S.failed, err);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(acc * np_pad);
                uint32_t accumulate = 0;
                for (int c = 0; c < nchunk; c++) {
                    int stage;
                    uint32_t phase;
                    ring_slot(acc, q[acc]++, stage, phase);
                    if (!mbar_wait(&S.full[stage], phase, TC_WAIT_CYCLES)) {
                        tc_fail(S.failed, err);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int sp = c / kc_n, kc = c % kc_n;
                    const uint32_t a0 = smem_u32(sA + stage * a_chunk);
                    const uint32_t bh = smem_u32(sB + kc * b_chunk);
                    const uint32_t bl = smem_u32(sB + (kc_n + kc) * b_chunk);
                    for (int k = 0; k < KW / 16; k++) {
                        mma_bf16(d, smem_desc_rows<RB>(a0 + 32 * k), smem_desc_rows<RB>(bh + 32 * k), idesc,
                                 accumulate);
                        accumulate = 1;
                    }
                    if (sp < 2)  // V_hi C_lo, V_mid C_lo (V_lo C_lo dropped)
                        for (int k = 0; k < KW / 16; k++)
                            mma_bf16(d, smem_desc_rows<RB>(a0 + 32 * k), smem_desc_rows<RB>(bl + 32 * k),
                                     idesc, 1);
                    mma_commit(&S.empty[stage]);
                }
                if (!ok) break;
                mma_commit(&S.tfull[acc]);
                if (++acc == 2) {
                    acc = 0;
                    aphase ^= 1;
                }
            }
        }
    } else {  // ------------------------------------------------ epilogue
        const int quarter = warp & 3;
        const int grp = (warp - 2) / TC_GROUP_WARPS;              // tiles i with i % 2 == grp
        const int split = ((warp - 2) % TC_GROUP_WARPS) >> 2;     // colour groups g % TC_NSPLIT
        const int m = quarter * 32 + lane;      // tile row this thread owns
        const int acc = grp;                    // the group's TMEM accumulator
        uint32_t aphase = 0;
        const int gsize = cpe < TC_M ? cpe : TC_M;   // rows of one event in a tile (power of two)
        const int wseg = gsize < 32 ? gsize : 32;    // lanes per warp segment
        const int spg = gsize / wseg;                // segments per event group
        const int ppt = TC_NSPLIT * (TC_M / wseg);   // partials per tile
        // partial of (tile t, group m / gsize, colour set, segment in group)
        const long long pidx0 = (long long)((m / gsize) * TC_NSPLIT + split) * spg + (m % gsize) / wseg;
        bool ok = true;
        long long i = grp;                      // index of the tile among this CTA's tiles
        for (long long t = blockIdx.x + grp * (long long)gridDim.x; ok && t < ntiles;
             t += TC_NGROUP * (long long)gridDim.x, i += TC_NGROUP) {
            float v[kp / TC_NSPLIT];            // v[16 (g / TC_NSPLIT) + j] = V of colour 16 g + j
#pragma unroll
            for (int c = 0; c < nchunk; c++) {
                int stage;
                uint32_t phase;
                ring_slot(grp, (i / TC_NGROUP) * nchunk + c, stage, phase);   // this group's ring
                if (ok)
                    ok = __all_sync(0xffffffffu, !*(volatile int *)S.failed &&
                                                     mbar_wait(&S.full[stage], phase, TC_WAIT_CYCLES));
                if (ok) {
                    const unsigned char *rowp = sA + stage * a_chunk + m * RB;
                    const int sp = c / kc_n, kc = c % kc_n;
#pragma unroll
                    for (int gg = 0; gg < GPC / TC_NSPLIT; gg++) {   // groups GPC kc + split + TC_NSPLIT gg
#pragma unroll
                        for (int pc = 0; pc < 2; pc++) {    // 8-colour pieces of the group
                            const int j = 2 * (split + TC_NSPLIT * gg) + pc;
                            // 16-byte piece j of row m: 128-byte swizzle at j ^ (m % 8),
                            // 64-byte swizzle at j ^ ((m / 2) % 4)
                            const int jp = RB == 128 ? (j ^ (m & 7)) : (j ^ ((m >> 1) & 3));
                            const uint4 q = *reinterpret_cast<const uint4 *>(rowp + (jp << 4));
                            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
                            float *d = &v[(kc * (GPC / TC_NSPLIT) + gg) * 16 + 8 * pc];
#pragma unroll
                            for (int i = 0; i < 4; i++) {
                                const float lo = __uint_as_float(w[i] << 16);
                                const float hi = __uint_as_float(w[i] & 0xFFFF0000u);
                                if (sp == 0) {
                                    d[2 * i] = lo;
                                    d[2 * i + 1] = hi;
                                } else {
                                    d[2 * i] += lo;
                                    d[2 * i + 1] += hi;
                                }
                            }
                        }
                    }
                    // the stage goes back to the TMA producer: this thread's
                    // shared-memory reads (generic proxy) must be complete
                    // before the next copy (async proxy) may overwrite it
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0)
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                         smem_u32(&S.empty[stage]))
                                     : "memory");
                }
            }
            if (ok)
                ok = __all_sync(0xffffffffu, !*(volatile int *)S.failed &&
                                                 mbar_wait(&S.tfull[acc], aphase, TC_WAIT_CYCLES));
            if (!ok) {
                if (lane == 0) tc_fail(S.failed, err);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t taddr = tmem + (uint32_t)(acc * np_pad) + ((uint32_t)(quarter * 32) << 16);
            float sh = 0.0f, sl = 0.0f;
#pragma unroll
            for (int gl = 0; gl < kp / (16 * TC_NSPLIT); gl++) {
                const int c0 = 16 * (TC_NSPLIT * gl + split);
                if (c0 < np) {   // colours >= np: zero columns of C_hat, Z = 0
                    uint32_t z[16];
                    tmem_ld16(taddr + (uint32_t)c0, z);
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const float vv = v[16 * gl + j];
                        const float zz = __uint_as_float(z[j]);
                        const float p = vv * zz;
                        const float pe = fmaf(vv, zz, -p);      // exact product p + pe
                        const float s = sh + p;                  // two-sum (sh, p)
                        const float bp = s - sh;
                        const float se = (sh - (s - bp)) + (p - bp);
                        sh = s;
                        sl += se + pe;
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&S.tempty[acc]))
                             : "memory");
            // butterfly over the warp segment (every lane ends with the same bits)
            double cs = (double)sh + (double)sl;
            for (int off = wseg >> 1; off >= 1; off >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, off);
            if ((lane & (wseg - 1)) == 0) part[t * ppt + pidx0] = cs;
            aphase ^= 1;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(tmem_cols)
                     : "memory");
    }
}

// me[e] = factor * (sum of the event's partial sums), fixed order: the
// partials of one event are contiguous (tile, event group, colour set,
// segment), per_event of them.
__global__ void k_event_sum(const double *__restrict__ part, long long nevt, int per_event,
                            double factor, double *__restrict__ me) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nevt) return;
    double s = 0.0;
    for (int j = 0; j < per_event; j++) s += part[e * per_event + j];
    me[e] = s * factor;
}

// ---------------------------------------------------------------------------
// Colour sum of the 5040-flow process on the tensor cores.  The quadratic
// form of every GEMM row V (3 BF16 pieces, KP colours) is taken over the
// block upper triangle of D*C in 128 x 128 blocks:
//   q_r = sum_I sum_{J >= I} w_IJ sum_{n in I} V_rn Z^(J)_rn,
//   Z^(J)_rn = sum_{k in J} C_hat_nk V_rk,  w_II = 1, w_IJ = 2 (J > I).
// Work item (M-tile of 128 rows, N-tile I), static round-robin over the
// CTAs.  Each K-block J (two 64-colour chunks: 3 A pieces + C_hi, C_lo halves,
// 80 KiB per chunk through a 2-stage ring) is accumulated in a fresh TMEM
// accumulator (two alternate), so FP32 accumulation spans 128 colours as in
// the single-tile kernel; the epilogue adds the blocks' dot products in FP64.
// Roles: warp 0 TMA producer, warp 1 MMA issuer (one thread), warps 2-9
// epilogue (lane quarter warp % 4, colour half (warp - 2) / 4 of the
// N-tile; its 64 values of V held in registers for the whole item, read
// once from the row buffer).  Writes part[(2 I + half) * R + r].
constexpr int TB_STAGES = 2;
constexpr int TB_CHUNK = 5 * TC_M * 128;          // bytes per K-chunk stage
constexpr int TB_THREADS = 64 + 32 * 8;

__global__ void __launch_bounds__(TB_THREADS, 1)
    k_colorsum_tc_big(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const __nv_bfloat16 *__restrict__ jb, int kp, int np, long long mtiles,
                      uint32_t extra_tx, double *__restrict__ part, long long R,
                      int *__restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + TB_STAGES * TB_CHUNK);
    uint64_t *empty = full + TB_STAGES;
    uint64_t *tfull = empty + TB_STAGES;
    uint64_t *tempty = tfull + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
    int *failed = reinterpret_cast<int *>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntile_n = np / TC_M;                 // N-tiles = K-blocks
    const long long nitems = mtiles * ntile_n;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int i = 0; i < TB_STAGES; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; i++) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], 8);
        }
        *failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // items in order: N-tile major (all CTAs share the colour-matrix band of one
    // N-tile in L2; taking them M-tile major halved the DRAM reads of the row
    // tiles but was 10% slower), M-tile minor
    if (warp == 0) {
        if (lane == 0) {  // ------------------------------------ producer
            long long cc = 0;   // chunk counter over the CTA's items
            bool ok = true;
            for (long long it = blockIdx.x; ok && it < nitems; it += gridDim.x) {
                const int I = (int)(it / mtiles);
                const long long t = it % mtiles;
                for (int kc = 2 * I; kc < 2 * ntile_n; kc++, cc++) {
                    const int st = (int)(cc % TB_STAGES);
                    const uint32_t ph = (uint32_t)((cc / TB_STAGES) & 1);
                    if (*(volatile int *)failed || !mbar_wait(&empty[st], ph ^ 1, TC_WAIT_CYCLES)) {
                        tc_fail(failed, err);
                        ok = false;
                        break;
                    }
                    unsigned char *dst = smem + st * TB_CHUNK;
                    mbar_expect_tx(&full[st], (uint32_t)TB_CHUNK + extra_tx);
                    for (int sp = 0; sp < 3; sp++)
                        tma_load_2d(dst + sp * TC_M * 128, &tmA, sp * kp + kc * TC_KCHUNK,
                                    (int)(t * TC_M), &full[st]);
                    for (int h = 0; h < 2; h++)
                        tma_load_2d(dst + (3 + h) * TC_M * 128, &tmB, kc * TC_KCHUNK,
                                    h * np + I * TC_M, &full[st]);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ------------------------------------ MMA issuer
            const uint32_t idesc = instr_desc(TC_M, TC_M);
            long long cc = 0, kb = 0;   // chunk and K-block counters
            bool ok = true;
            for (long long it = blockIdx.x; ok && it < nitems; it += gridDim.x) {
                const int I = (int)(it / mtiles);
                for (int J = I; ok && J < ntile_n; J++, kb++) {
                    const int acc = (int)(kb & 1);
                    const uint32_t aph = (uint32_t)((kb >> 1) & 1);
                    if (*(volatile int *)failed || !mbar_wait(&tempty[acc], aph ^ 1, TC_WAIT_CYCLES)) {
                        tc_fail(failed, err);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t d = tmem + (uint32_t)(acc * TC_M);
                    uint32_t accumulate = 0;
                    for (int h = 0; h < 2; h++, cc++) {   // the block's two K-chunks
                        const int st = (int)(cc % TB_STAGES);
                        const uint32_t ph = (uint32_t)((cc / TB_STAGES) & 1);
                        if (!mbar_wait(&full[st], ph, TC_WAIT_CYCLES)) {
                            tc_fail(failed, err);
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t base = smem_u32(smem + st * TB_CHUNK);
                        const uint32_t bh = base + 3 * TC_M * 128, bl = base + 4 * TC_M * 128;
                        for (int sp = 0; sp < 3; sp++) {
                            const uint32_t a0 = base + sp * TC_M * 128;
                            for (int k = 0; k < TC_KCHUNK / 16; k++) {
                                mma_bf16(d, smem_desc(a0 + 32 * k), smem_desc(bh + 32 * k), idesc, accumulate);
                                accumulate = 1;
                            }
                            if (sp < 2)
                                for (int k = 0; k < TC_KCHUNK / 16; k++)
                                    mma_bf16(d, smem_desc(a0 + 32 * k), smem_desc(bl + 32 * k), idesc, 1);
                        }
                        mma_commit(&empty[st]);
                    }
                    if (!ok) break;
                    mma_commit(&tfull[acc]);
                }
            }
        }
    } else {  // ------------------------------------------------ epilogue
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int m = quarter * 32 + lane;
        long long kb = 0;
        bool ok = true;
        for (long long it = blockIdx.x; ok && it < nitems; it += gridDim.x) {
            const int I = (int)(it / mtiles);
            const long long t = it % mtiles;
            const long long r = t * TC_M + m;
            // V of this row on the 64 colours of the N-tile half, hi + mid + lo
            float v[64];
            const __nv_bfloat16 *row = jb + r * (long long)(3 * kp) + I * TC_M + half * 64;
#pragma unroll
            for (int c8 = 0; c8 < 8; c8++) {
                uint4 q[3];
#pragma unroll
                for (int sp = 0; sp < 3; sp++) q[sp] = *reinterpret_cast<const uint4 *>(row + sp * kp + 8 * c8);
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    float lo = 0.0f, hi = 0.0f;
#pragma unroll
                    for (int sp = 0; sp < 3; sp++) {
                        const uint32_t w = (&q[sp].x)[i];
                        lo += __uint_as_float(w << 16);
                        hi += __uint_as_float(w & 0xFFFF0000u);
                    }
                    v[8 * c8 + 2 * i] = lo;
                    v[8 * c8 + 2 * i + 1] = hi;
                }
            }
            double total = 0.0;
            for (int J = I; J < ntile_n; J++, kb++) {
                const int acc = (int)(kb & 1);
                const uint32_t aph = (uint32_t)((kb >> 1) & 1);
                ok = __all_sync(0xffffffffu, !*(volatile int *)failed &&
                                                 mbar_wait(&tfull[acc], aph, TC_WAIT_CYCLES));
                if (!ok) {
                    if (lane == 0) tc_fail(failed, err);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t taddr = tmem + (uint32_t)(acc * TC_M + half * 64) + ((uint32_t)(quarter * 32) << 16);
                float sh = 0.0f, sl = 0.0f;
#pragma unroll
                for (int g = 0; g < 4; g++) {
                    uint32_t z[16];
                    tmem_ld16(taddr + (uint32_t)(16 * g), z);
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const float vv = v[16 * g + j];
                        const float zz = __uint_as_float(z[j]);
                        const float p = vv * zz;
                        const float pe = fmaf(vv, zz, -p);
                        const float s = sh + p;
                        const float bp = s - sh;
                        const float se = (sh - (s - bp)) + (p - bp);
                        sh = s;
                        sl += se + pe;
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[acc]))
                                 : "memory");
                total += (J == I ? 1.0 : 2.0) * ((double)sh + (double)sl);
            }
            if (!ok) break;
            part[(long long)(2 * I + half) * R + r] = total;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256)
                     : "memory");
    }
}

// me[e] = factor * sum over the event's cpe rows (contiguous from e * cpe)
// and the ncols partial columns part[c * R + r], in that fixed order.
__global__ void k_event_sum_rows(const double *__restrict__ part, long long R, int ncols, int cpe,
                                 long long nevt, double factor, double *__restrict__ me) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nevt) return;
    double s = 0.0;
    for (int j = 0; j < cpe; j++)
        for (int c = 0; c < ncols; c++) s += part[(long long)c * R + e * cpe + j];
    me[e] = s * factor;
}

// Caller rows to tensor-core rows (test hook): rows[r * nc + c] (FP64) to
// jb[r * 3 kp + s * kp + c] as three BF16 pieces (the value rounded to FP32,
// then split twice), colours >= nc zero.
__global__ void k_rows_split(const double *__restrict__ rows, long long nrows, int nc, int kp,
                             __nv_bfloat16 *__restrict__ jb) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nrows * kp) return;
    const long long r = idx / kp;
    const int c = (int)(idx % kp);
    const float f = c < nc ? __double2float_rn(rows[r * nc + c]) : 0.0f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(f);
    const float r1 = f - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    __nv_bfloat16 *row = jb + r * (long long)(3 * kp);
    row[c] = hi;
    row[kp + c] = mid;
    row[2 * kp + c] = __float2bfloat16_rn(r1 - __bfloat162float(mid));
}

}  // namespace

int mg_tc_parts_per_tile(int cpe) {
    const int gsize = cpe < TC_M ? cpe : TC_M;
    return TC_NSPLIT * (TC_M / (gsize < 32 ? gsize : 32));
}

int mg_tc_parts_per_event(int cpe) {
    const int gsize = cpe < TC_M ? cpe : TC_M;
    const int tiles = cpe > TC_M ? cpe / TC_M : 1;
    return tiles * TC_NSPLIT * (gsize / (gsize < 32 ? gsize : 32));
}

size_t mg_tc_smem_bytes(int kp, int np) {
    const int kw = kp == 32 ? 32 : TC_KCHUNK;   // colours per chunk
    const int kc_n = kp / kw;
    return 1024 + (size_t)2 * kc_n * np * 2 * kw + (size_t)TC_STAGES * TC_M * 2 * kw +
           (1 + 2 * TC_STAGES + 4) * 8 + 16;
}

cudaError_t mg_launch_colorsum_tc(const __nv_bfloat16 *jbuf, long long ncols_alloc, int kp,
                                  const __nv_bfloat16 *cmat, int np, int ncolor, int cpe,
                                  uint32_t extra_tx, double *part, int *err, cudaStream_t stream) {
    if (ncols_alloc % TC_M || (kp != 32 && kp != TC_KCHUNK && kp != 2 * TC_KCHUNK) || np % 16 ||
        np > 128 || np > kp || cpe < 8 || (cpe & (cpe - 1)))
        return cudaErrorInvalidValue;
    const uint32_t kw = kp == 32 ? 32u : (uint32_t)TC_KCHUNK;   // colours per chunk
    CUtensorMap ma, mb;
    if (!make_map(&ma, jbuf, (uint64_t)ncols_alloc, (uint64_t)3 * kp, TC_M, kw)) return cudaErrorInvalidValue;
    if (!make_map(&mb, cmat, (uint64_t)2 * np, (uint64_t)kp, (uint32_t)np, kw)) return cudaErrorInvalidValue;
    int np_pad = 32;
    while (np_pad < np) np_pad <<= 1;
    const int tmem_cols = 2 * np_pad;  // two accumulators
    const size_t smem = mg_tc_smem_bytes(kp, np);
    cudaError_t e =
        kp == 32 ? cudaFuncSetAttribute(k_colorsum_tc<32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem)
        : kp == TC_KCHUNK
            ? cudaFuncSetAttribute(k_colorsum_tc<TC_KCHUNK, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem)
            : cudaFuncSetAttribute(k_colorsum_tc<TC_KCHUNK, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const long long ntiles = ncols_alloc / TC_M;
    const long long grid = ntiles < nsm ? ntiles : nsm;   // persistent: one CTA per SM
    mg_note_launch();
    if (kp == 32)
        k_colorsum_tc<32, 1><<<(unsigned)grid, TC_THREADS, smem, stream>>>(ma, mb, np, np_pad, cpe, ntiles,
                                                                           tmem_cols, extra_tx, part, err);
    else if (kp == TC_KCHUNK)
        k_colorsum_tc<TC_KCHUNK, 1><<<(unsigned)grid, TC_THREADS, smem, stream>>>(
            ma, mb, np, np_pad, cpe, ntiles, tmem_cols, extra_tx, part, err);
    else
        k_colorsum_tc<TC_KCHUNK, 2><<<(unsigned)grid, TC_THREADS, smem, stream>>>(
            ma, mb, np, np_pad, cpe, ntiles, tmem_cols, extra_tx, part, err);
    return cudaGetLastError();
}

size_t mg_tc_big_smem_bytes() { return 1024 + (size_t)TB_STAGES * TB_CHUNK + (4 * TB_STAGES + 4) * 8 + 16; }

cudaError_t mg_launch_colorsum_tc_big(const __nv_bfloat16 *jb, long long R, int kp,
                                      const __nv_bfloat16 *cmat, int np, uint32_t extra_tx,
                                      double *part, int *err, cudaStream_t stream) {
    if (R <= 0) return cudaSuccess;
    if (R % TC_M || kp % TC_M || np != kp) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map(&ma, jb, (uint64_t)R, (uint64_t)3 * kp, TC_M)) return cudaErrorInvalidValue;
    if (!make_map(&mb, cmat, (uint64_t)2 * np, (uint64_t)kp, TC_M)) return cudaErrorInvalidValue;
    const size_t smem = mg_tc_big_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_colorsum_tc_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const long long mtiles = R / TC_M;
    const long long nitems = mtiles * (np / TC_M);
    const long long grid = nitems < nsm ? nitems : nsm;
    mg_note_launch();
    k_colorsum_tc_big<<<(unsigned)grid, TB_THREADS, smem, stream>>>(ma, mb, jb, kp, np, mtiles, extra_tx,
                                                                     part, R, err);
    return cudaGetLastError();
}

cudaError_t mg_launch_rows_split(const double *rows, long long nrows, int nc, int kp,
                                 __nv_bfloat16 *jb, cudaStream_t stream) {
    if (nrows <= 0) return cudaSuccess;
    const long long n = nrows * kp;
    mg_note_launch();
    k_rows_split<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(rows, nrows, nc, kp, jb);
    return cudaGetLastError();
}

cudaError_t mg_launch_event_sum_rows(const double *part, long long R, int ncols, int cpe, long long nevt,
                                     double factor, double *me, cudaStream_t stream) {
    if (nevt <= 0) return cudaSuccess;
    if (nevt * cpe > R) return cudaErrorInvalidValue;
    mg_note_launch();
    k_event_sum_rows<<<(unsigned)((nevt + 127) / 128), 128, 0, stream>>>(part, R, ncols, cpe, nevt, factor, me);
    return cudaGetLastError();
}

cudaError_t mg_launch_event_sum(const double *part, long long nevt, int per_event, double factor,
                                double *me, cudaStream_t stream) {
    if (nevt <= 0) return cudaSuccess;
    mg_note_launch();
    k_event_sum<<<(unsigned)((nevt + 255) / 256), 256, 0, stream>>>(part, nevt, per_event, factor, me);
    return cudaGetLastError();
}
