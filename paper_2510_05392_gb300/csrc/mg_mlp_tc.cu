// GEMMs of the surrogate MLP on the tensor cores (tcgen05, sm_103a).
//
// Every contraction of the network's forward and backward passes is
//   D[m][n] = sum_k X[m][k] Y[n][k]
// with X and Y row-major BF16 (K contiguous), brought to shared memory by
// TMA (cp.async.bulk.tensor, 128-byte swizzle, 64-wide K chunks; parts of a
// box outside the tensor are filled with zeros), multiplied by
// tcgen05.mma kind::f16 (M = 128, N = the CTA's column tile, K = 16) into an
// FP32 accumulator in tensor memory, and finished by a fused epilogue:
//   forward hidden layer  X = A_l [batch][in], Y = W_l [out][in]:
//                         z = D + b, Z = z (FP32), A_l+1 = silu(z) (BF16,
//                         row-major and transposed)
//   forward output layer  z = D + b (FP32)
//   backward data         X = dZ_l [batch][out], Y = W_l^T [in][out]:
//                         dZ_l-1 = D * silu'(Z_l-1) (BF16 row-major and
//                         transposed, FP32 copy for the bias gradient)
//   weight gradient       X = dZ_l^T [out][batch], Y = A_l^T [in][batch]:
//                         partial sums of gW_l = D over a slice of the batch
//                         (split K, summed in a fixed order afterwards)
// Roles (128 threads): warp 0 lane 0 loads the stages by TMA, warp 1 lane 0
// issues the MMAs and commits; after the last commit all four warps read the
// accumulator (thread t owns row t: TMEM lane t) and run the epilogue.  Every
// mbarrier wait is bounded; on timeout the CTA records MG_TC_ERR_TIMEOUT in
// *err, skips its stores, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mg_internal.h"
#include "mg_mlp.h"
#include "mg_tc.cuh"

namespace {

using namespace mgtc;

constexpr int ML_STAGES = 4;
constexpr int ML_THREADS = 128;
constexpr int ML_X_BYTES = TC_M * 128;   // one 128-row x 64-K chunk of X

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

template <int MODE>
__global__ void __launch_bounds__(ML_THREADS, 1)
    k_mlp_gemm(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
               int nt, int kchunks, int tmem_cols, uint32_t extra_tx, mg_mlp_epi ep,
               int *__restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int y_bytes = nt * 128;
    const int stage_bytes = ML_X_BYTES + y_bytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + ML_STAGES * stage_bytes);
    uint64_t *empty = full + ML_STAGES;
    uint64_t *tfull = empty + ML_STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tfull + 1);
    int *failed = reinterpret_cast<int *>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * nt;
    const int kc0 = blockIdx.z * kchunks;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int i = 0; i < ML_STAGES; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(tfull, 1);
        *failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {  // ---------------------------- producer
        for (int c = 0; c < kchunks; c++) {
            const int s = c % ML_STAGES;
            const uint32_t ph = (uint32_t)((c / ML_STAGES) & 1);
            if (!mbar_wait(&empty[s], ph ^ 1, TC_WAIT_CYCLES)) {
                atomicExch(failed, 1);
                atomicExch(err, MG_TC_ERR_TIMEOUT);
                break;
            }
            unsigned char *dst = smem + s * stage_bytes;
            mbar_expect_tx(&full[s], (uint32_t)stage_bytes + extra_tx);
            tma_load_2d(dst, &tmX, (kc0 + c) * TC_KCHUNK, m0, &full[s]);
            tma_load_2d(dst + ML_X_BYTES, &tmY, (kc0 + c) * TC_KCHUNK, n0, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {  // ------------------- MMA issuer
        const uint32_t idesc = instr_desc(TC_M, nt);
        bool ok = true;
        for (int c = 0; c < kchunks && ok; c++) {
            const int s = c % ML_STAGES;
            const uint32_t ph = (uint32_t)((c / ML_STAGES) & 1);
            if (!mbar_wait(&full[s], ph, TC_WAIT_CYCLES) || *(volatile int *)failed) {
                atomicExch(failed, 1);
                atomicExch(err, MG_TC_ERR_TIMEOUT);
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(smem + s * stage_bytes);
            const uint32_t b0 = a0 + ML_X_BYTES;
#pragma unroll
            for (int k = 0; k < TC_KCHUNK / 16; k++)
                mma_bf16(tmem, smem_desc(a0 + 32 * k), smem_desc(b0 + 32 * k), idesc,
                         (c > 0 || k > 0) ? 1u : 0u);
            mma_commit(&empty[s]);
        }
        if (ok) mma_commit(tfull);
    }
    __syncwarp();
    // ------------------------------------------------------------ epilogue
    const bool ok = mbar_wait(tfull, 0, TC_WAIT_CYCLES) && !*(volatile int *)failed;
    if (!ok && lane == 0) {
        atomicExch(failed, 1);
        atomicExch(err, MG_TC_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int m = m0 + tid;                                    // this thread's row (TMEM lane tid)
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    if (__all_sync(0xffffffffu, ok)) {
        for (int c0 = 0; c0 < nt; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(taddr + (uint32_t)c0, r);
            const int n = n0 + c0;
            if (m >= ep.m_valid) continue;
            if constexpr (MODE == MG_MLP_WGRAD) {
                float *dst = ep.part + ((long long)blockIdx.z * ep.m_valid + m) * ep.ldz + n;
#pragma unroll
                for (int j = 0; j < 16; j++)
                    if (n + j < ep.n_valid) dst[j] = __uint_as_float(r[j]);
            } else {
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
                const long long o = (long long)m * ep.ldz + n;
                if constexpr (MODE == MG_MLP_FWD || MODE == MG_MLP_FWD_OUT) {
#pragma unroll
                    for (int j = 0; j < 16; j++) v[j] += __ldg(ep.bias + n + j);
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        *reinterpret_cast<float4 *>(ep.Z + o + 4 * q) =
                            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    if constexpr (MODE == MG_MLP_FWD) {
                        __align__(16) __nv_bfloat16 a[16];
#pragma unroll
                        for (int j = 0; j < 16; j++) a[j] = __float2bfloat16_rn(silu_f(v[j]));
                        *reinterpret_cast<uint4 *>(ep.A + o) = *reinterpret_cast<const uint4 *>(a);
                        *reinterpret_cast<uint4 *>(ep.A + o + 8) = *reinterpret_cast<const uint4 *>(a + 8);
#pragma unroll
                        for (int j = 0; j < 16; j++) ep.AT[(long long)(n + j) * ep.ldt + m] = a[j];
                    }
                } else {  // MG_MLP_BWD_DATA
                    __align__(16) __nv_bfloat16 d16[16];
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        v[j] *= dsilu_f(__ldg(ep.Zprev + o + j));
                        d16[j] = __float2bfloat16_rn(v[j]);
                    }
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        *reinterpret_cast<float4 *>(ep.dZ32 + o + 4 * q) =
                            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    *reinterpret_cast<uint4 *>(ep.dZ + o) = *reinterpret_cast<const uint4 *>(d16);
                    *reinterpret_cast<uint4 *>(ep.dZ + o + 8) = *reinterpret_cast<const uint4 *>(d16 + 8);
#pragma unroll
                    for (int j = 0; j < 16; j++) ep.dZT[(long long)(n + j) * ep.ldt + m] = d16[j];
                }
            }
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

size_t ml_smem_bytes(int nt) { return 1024 + (size_t)ML_STAGES * (ML_X_BYTES + nt * 128) + (2 * ML_STAGES + 1) * 8 + 16; }

// 2-D BF16 tensor map [rows][cols] with row stride ld elements, box 64 x box_rows,
// 128-byte swizzle; parts of a box outside the tensor read as zeros.
bool make_map_ld(CUtensorMap *m, const void *base, uint64_t rows, uint64_t cols, uint64_t ld,
                 uint32_t box_rows) {
    encode_tiled_fn f = encode_fn();
    if (!f) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TC_KCHUNK, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return f(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t mg_launch_mlp_gemm(int mode, const __nv_bfloat16 *X, long long xrows, long long xld,
                               const __nv_bfloat16 *Y, long long yrows, long long yld, int kdim,
                               long long M, int N, int nt, int ksplit, const mg_mlp_epi &ep, int *err,
                               cudaStream_t stream, uint32_t extra_tx) {
    // M rows of D in 128-row tiles, N columns in nt-column tiles, K = kdim
    // in 64-wide chunks, split in ksplit equal slices (weight gradient only);
    // TMA needs 16-byte row strides and a 16-byte aligned base
    if (M <= 0 || M % TC_M || N % nt || nt < 16 || nt > 256 || nt % 16 || kdim < 1 || ksplit < 1 ||
        xld % 8 || yld % 8 || xld < kdim || yld < kdim || xrows < 1 || yrows < 1 ||
        (reinterpret_cast<uintptr_t>(X) & 15) || (reinterpret_cast<uintptr_t>(Y) & 15))
        return cudaErrorInvalidValue;
    const int kch = (kdim + TC_KCHUNK - 1) / TC_KCHUNK;
    if (kch % ksplit || (mode != MG_MLP_WGRAD && ksplit != 1)) return cudaErrorInvalidValue;
    CUtensorMap mx, my;
    if (!make_map_ld(&mx, X, (uint64_t)xrows, (uint64_t)kdim, (uint64_t)xld, TC_M))
        return cudaErrorInvalidValue;
    if (!make_map_ld(&my, Y, (uint64_t)yrows, (uint64_t)kdim, (uint64_t)yld, (uint32_t)nt))
        return cudaErrorInvalidValue;
    int tmem_cols = 32;
    while (tmem_cols < nt) tmem_cols <<= 1;
    const size_t smem = ml_smem_bytes(nt);
    const dim3 grid((unsigned)(M / TC_M), (unsigned)(N / nt), (unsigned)ksplit);
    // the dynamic shared-memory limit of each mode, raised once per device
    // (a host call per launch would cost as much as the launch itself)
    static size_t smem_set[64][4];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool raise = dev < 0 || dev >= 64 || mode < 0 || mode > 3 || smem_set[dev][mode] < smem;
    mg_note_launch();
    switch (mode) {
#define ML_CASE(MD)                                                                                \
    case MD:                                                                                       \
        if (raise) {                                                                               \
            e = cudaFuncSetAttribute(k_mlp_gemm<MD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
            if (e != cudaSuccess) return e;                                                        \
            if (dev >= 0 && dev < 64) smem_set[dev][MD] = smem;                                    \
        }                                                                                          \
        k_mlp_gemm<MD><<<grid, ML_THREADS, smem, stream>>>(mx, my, nt, kch / ksplit, tmem_cols, extra_tx, ep, \
                                                           err);                                   \
        break;
        ML_CASE(MG_MLP_FWD)
        ML_CASE(MG_MLP_FWD_OUT)
        ML_CASE(MG_MLP_BWD_DATA)
        ML_CASE(MG_MLP_WGRAD)
#undef ML_CASE
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
