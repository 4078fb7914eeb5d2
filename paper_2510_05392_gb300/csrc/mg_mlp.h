// Tensor-core GEMMs of the surrogate MLP (mg_mlp_tc.cu), used by
// mg_surrogate.cu.  D[m][n] = sum_k X[m][k] Y[n][k], X and Y row-major BF16
// with K contiguous, FP32 accumulation, fused epilogue by mode.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

enum {
    MG_MLP_FWD = 0,       // z = D + b -> Z (FP32), A = silu(z) (BF16) and its transpose AT
    MG_MLP_FWD_OUT = 1,   // z = D + b -> Z (FP32)
    MG_MLP_BWD_DATA = 2,  // d = D * silu'(Zprev) -> dZ (BF16), its transpose dZT, dZ32 (FP32)
    MG_MLP_WGRAD = 3      // part[split][m][n] = D over the split's slice of K (FP32)
};

typedef struct {
    const float *bias;       // [N]                     (forward)
    float *Z;                // [rows][ldz]             (forward)
    __nv_bfloat16 *A;        // [rows][ldz]             (forward, hidden)
    __nv_bfloat16 *AT;       // [ldz][ldt]              (forward, hidden)
    const float *Zprev;      // [rows][ldz]             (backward data)
    __nv_bfloat16 *dZ;       // [rows][ldz]             (backward data)
    __nv_bfloat16 *dZT;      // [ldz][ldt]              (backward data)
    float *dZ32;             // [rows][ldz]             (backward data)
    float *part;             // [split][m_valid][ldz]   (weight gradient)
    int ldz;                 // columns of the row-major outputs
    long long ldt;           // columns of the transposed outputs (rows of the batch buffer)
    int m_valid, n_valid;    // rows (and, weight gradient, columns) that are written
} mg_mlp_epi;

// X: xrows rows of row stride xld; Y: yrows rows of row stride yld; K = kdim
// (64-wide chunks, zero-filled past kdim and past the last row); D is M x N
// (M multiple of 128, N multiple of nt, nt in 16..256 a multiple of 16);
// ksplit slices of K (weight gradient only).  err: device word set to
// MG_TC_ERR_TIMEOUT when a bounded wait gives up.  extra_tx (test hook): bytes
// the operand barrier expects beyond what arrives (0 in normal use).
cudaError_t mg_launch_mlp_gemm(int mode, const __nv_bfloat16 *X, long long xrows, long long xld,
                               const __nv_bfloat16 *Y, long long yrows, long long yld, int kdim,
                               long long M, int N, int nt, int ksplit, const mg_mlp_epi &ep, int *err,
                               cudaStream_t stream, uint32_t extra_tx = 0);
