// MLP surrogate of log|M|^2 and the two-stage unweighting it drives.
//
// The paper has no learned component; this is the benchmark configuration's
// surrogate pattern, the published scheme of rejection sampling with network
// weight estimates (Danziger, Janssen, Schumann, Siegert 2022):
//   features  x = log(s_ij / s) over all particle pairs (FP64, rounded to BF16)
//   network   z_1 = W_1 x + b_1, a = silu(z), ..., f = z_L;  sizes
//             nin -> hidden (x nhidden, SiLU) -> 1; BF16 weights/activations,
//             FP32 accumulation, FP32 master weights, Adam
//   target    y = (log|M|^2 - mu) / sigma, MSE loss
//   unweight  w_hat = exp(sigma f + mu) Phi; stage 1 keeps u1 < w_hat/w_hat_max;
//             the exact FP64 matrix element is evaluated for those only;
//             stage 2 keeps u2 < (w/w_hat)/r_max, w = |M|^2 Phi; weight
//             max(1, w_hat/w_hat_max) * max(1, (w/w_hat)/r_max)
// GEMMs run on the 5th-generation tensor cores (mg_mlp_tc.cu: tcgen05.mma
// with TMA-fed shared-memory operands and FP32 accumulators in tensor
// memory) with bias / SiLU / SiLU' fused into their epilogues; the weight
// gradients are split over the batch and summed in a fixed order.  Every
// batch is padded to a multiple of 128 rows (zero features, zero loss
// gradient), so results do not depend on the padding.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "mg_mlp.h"
#include "mg_process.h"
#include "mgpu.h"
#include "mgpu_bench.h"
#include "mgpu_surrogate.h"

namespace {

constexpr int SUR_MAXL = 8;
constexpr int WM = 16;     // padding of layer widths
constexpr int MROWS = 128; // padding of batches (rows of one tensor-core tile)

// features: x[e][k] = log(s_ij / s) for pairs i < j (k in pair order): the
// ratio in FP64, its logarithm in FP32 (a BF16 input needs 8 bits; an FP64
// logarithm would cost ~40 instructions of the slow FP64 pipe per pair),
// rounded to BF16; zero padded, rows e >= n zero; written row-major [M][nin]
// and transposed [nin][ldt]
__global__ void k_features(const double *__restrict__ mom, long long n, long long M, int npar, int nin,
                           __nv_bfloat16 *__restrict__ x, __nv_bfloat16 *__restrict__ xt, long long ldt,
                           const int *__restrict__ bidx = nullptr) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M) return;
    if (bidx) mom += (long long)(*bidx) * n * npar * 4;   // batch *bidx of n rows
    int k = 0;
    if (e < n) {
        const double *p = mom + e * npar * 4;
        const double P0 = p[0] + p[4], P1 = p[1] + p[5], P2 = p[2] + p[6], P3 = p[3] + p[7];
        const double s = P0 * P0 - P1 * P1 - P2 * P2 - P3 * P3;
        for (int i = 0; i < npar; i++)
            for (int j = i + 1; j < npar; j++) {
                const double q0 = p[4 * i] + p[4 * j], q1 = p[4 * i + 1] + p[4 * j + 1];
                const double q2 = p[4 * i + 2] + p[4 * j + 2], q3 = p[4 * i + 3] + p[4 * j + 3];
                if (k < nin) {
                    const __nv_bfloat16 v =
                        __float2bfloat16_rn(logf((float)((q0 * q0 - q1 * q1 - q2 * q2 - q3 * q3) / s)));
                    x[e * nin + k] = v;
                    xt[(long long)k * ldt + e] = v;
                }
                k++;
            }
    }
    for (; k < nin; k++) {
        x[e * nin + k] = __float2bfloat16_rn(0.0f);
        xt[(long long)k * ldt + e] = __float2bfloat16_rn(0.0f);
    }
}

// Bias gradient gb[n] = sum_m dZ[m][n] from the FP32 values (the BF16 copies
// feed the weight-gradient GEMM; their rounding would not cancel in this
// sum), in two fixed-order levels: k_bias_part sums 128-row chunks (block:
// 32 columns x 8 row slices of 16 rows, FP64), k_wgrad_reduce adds the chunks.
constexpr int BIAS_ROWS = 128;
__global__ void k_bias_part(const float *__restrict__ dZ, long long M, int N, double *__restrict__ bpart) {
    __shared__ double red[8][32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + tx;
    const long long m0 = (long long)blockIdx.y * BIAS_ROWS;
    double s = 0.0;
    if (n < N) {
#pragma unroll
        for (int r = ty; r < BIAS_ROWS; r += 8)
            if (m0 + r < M) s += dZ[(m0 + r) * N + n];
    }
    red[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && n < N) {
        double t = 0.0;
        for (int k = 0; k < 8; k++) t += red[k][tx];
        bpart[(long long)blockIdx.y * N + n] = t;
    }
}

// gW[i] = sum over the splits of the weight-gradient partials, and (i < nb)
// gb[i] = sum over the row chunks of the bias partials, both in a fixed order
__global__ void k_wgrad_reduce(const float *__restrict__ part, int nsplit, long long n,
                               float *__restrict__ gW, const double *__restrict__ bpart, int nchunk,
                               int nb, float *__restrict__ gb) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        float s = 0.0f;
        for (int k = 0; k < nsplit; k++) s += part[(long long)k * n + i];
        gW[i] = s;
    }
    if (i < nb) {
        double t = 0.0;
        for (int k = 0; k < nchunk; k++) t += bpart[(long long)k * nb + i];
        gb[i] = (float)t;
    }
}

// Output-layer loss gradient: dZ[m][0] = 2 (f_m - y_m) / nvalid for rows
// m < nvalid, 0 elsewhere (padded columns and rows), row-major [M][N], its
// transpose [N][ldt] and an FP32 copy; per-block partial sums of the squared
// error.
__global__ void k_loss(const float *__restrict__ Zout, long long M, int nvalid, int N,
                       const float *__restrict__ y, __nv_bfloat16 *__restrict__ dZ,
                       __nv_bfloat16 *__restrict__ dZT, long long ldt, float *__restrict__ dZ32,
                       double *__restrict__ part) {
    __shared__ double red[256];
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double se = 0.0;
    if (m < M) {
        float g = 0.0f;
        if (m < nvalid) {
            const float d = Zout[m * N] - y[m];
            se = (double)d * d;
            g = 2.0f * d / nvalid;
        }
        for (int c = 0; c < N; c++) {
            const float v = c == 0 ? g : 0.0f;
            dZ[m * N + c] = __float2bfloat16_rn(v);
            dZT[(long long)c * ldt + m] = __float2bfloat16_rn(v);
            dZ32[m * N + c] = v;
        }
    }
    red[threadIdx.x] = se;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Adam on FP32 master parameters [rows][cols] (rows >= the real output width
// of a padded layer stay zero: their gradients are zero); BF16 copies
// refreshed, row-major and (when given) transposed [cols][rows].
__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, __nv_bfloat16 *__restrict__ p16,
                       __nv_bfloat16 *__restrict__ p16t, int rows, int cols, float lr, float b1,
                       float b2, float eps, float c1, float c2,
                       const int *__restrict__ steps = nullptr) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * cols) return;
    if (steps) {  // bias corrections of step *steps + 1, from the device-side step count
        const float t = (float)(*steps + 1);
        c1 = 1.0f - powf(b1, t);
        c2 = 1.0f - powf(b2, t);
    }
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float w = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = w;
    if (p16) p16[i] = __float2bfloat16_rn(w);
    if (p16t) p16t[(i % cols) * rows + i / cols] = __float2bfloat16_rn(w);
}

// target: y = (log me - mu) / sigma, with mu/sigma from k_logstats (of
// batch *bidx of n rows when bidx is given)
__global__ void k_target(const double *__restrict__ me, long long n, const double *__restrict__ ms,
                         float *__restrict__ y, const int *__restrict__ bidx = nullptr) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (bidx) me += (long long)(*bidx) * n;
    if (i < n) y[i] = (float)((log(me[i]) - ms[0]) / ms[1]);
}

// device-side training state: [0] batch index within the epoch, [1] Adam
// steps taken; advanced once per training step
__global__ void k_step_advance(int *__restrict__ st) {
    st[0] += 1;
    st[1] += 1;
}

// acc += sum of a batch's loss partial sums, in a fixed order
__global__ void k_loss_acc(const double *__restrict__ part, int nb, double *__restrict__ acc) {
    double t = 0.0;
    for (int b = 0; b < nb; b++) t += part[b];
    acc[0] += t;
}

// mean and standard deviation of log(me) (single block, fixed order)
__global__ void k_logstats(const double *__restrict__ me, long long n, double *__restrict__ ms) {
    __shared__ double s1[256], s2[256];
    double a = 0.0, b = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const double l = log(me[i]);
        a += l;
        b += l * l;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            s1[threadIdx.x] += s1[threadIdx.x + s];
            s2[threadIdx.x] += s2[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mu = s1[0] / n;
        const double var = s2[0] / n - mu * mu;
        ms[0] = mu;
        ms[1] = var > 0 ? sqrt(var) : 1.0;
    }
}

// log|M|^2 prediction: sigma f + mu
__global__ void k_pred(const float *__restrict__ Zout, int N, long long n, const double *__restrict__ ms,
                       double *__restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ms[1] * (double)Zout[i * N] + ms[0];
}

// stage 1: w_hat = exp(logme_hat) Phi, flag u1 < w_hat / w_hat_max; block counts
__global__ void k_stage1(const double *__restrict__ logme_hat, const double *__restrict__ phi,
                         const double *__restrict__ u1, long long n, double what_max,
                         double *__restrict__ what, unsigned char *__restrict__ flag,
                         int *__restrict__ bcount) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double w = exp(logme_hat[i]) * phi[i];
        what[i] = w;
        const unsigned char f = u1[i] < w / what_max;
        flag[i] = f;
        if (f) atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) bcount[blockIdx.x] = cnt;
}

// exclusive scan of block counts (single block, fixed order)
__global__ void k_scan(int *__restrict__ bcount, int nb, long long *__restrict__ total) {
    if (threadIdx.x != 0) return;
    long long s = 0;
    for (int b = 0; b < nb; b++) {
        const int c = bcount[b];
        bcount[b] = (int)s;
        s += c;
    }
    *total = s;
}

// ordered compaction of stage-1 survivors; gathers their momenta
__global__ void k_compact(const unsigned char *__restrict__ flag, const int *__restrict__ boff,
                          long long n, const double *__restrict__ mom, int npar,
                          long long *__restrict__ idx, double *__restrict__ mom_out) {
    __shared__ int pos[1024];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int f = (i < n) ? flag[i] : 0;
    pos[threadIdx.x] = f;
    __syncthreads();
    if (threadIdx.x == 0) {  // fixed-order prefix inside the block
        int s = 0;
        for (int t = 0; t < (int)blockDim.x; t++) {
            const int v = pos[t];
            pos[t] = s;
            s += v;
        }
    }
    __syncthreads();
    if (f) {
        const long long o = boff[blockIdx.x] + pos[threadIdx.x];
        idx[o] = i;
        for (int k = 0; k < npar * 4; k++) mom_out[o * npar * 4 + k] = mom[i * npar * 4 + k];
    }
}

// stage 2 on the survivors: keep u2 < (w / w_hat) / r_max; weights
__global__ void k_stage2(const long long *__restrict__ idx, const double *__restrict__ me_exact,
                         long long m, const double *__restrict__ phi, const double *__restrict__ what,
                         const double *__restrict__ u2, double what_max, double r_max,
                         unsigned char *__restrict__ accept, double *__restrict__ weight) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const long long i = idx[k];
    const double w = me_exact[k] * phi[i];
    const double r = w / what[i];
    const bool a = u2[i] < r / r_max;
    accept[i] = a;
    const double w1 = what[i] / what_max;
    weight[i] = a ? fmax(1.0, w1) * fmax(1.0, r / r_max) : 0.0;
}

}  // namespace

struct mg_surrogate {
    int nl;                      // linear layers
    int in[SUR_MAXL], out[SUR_MAXL], outp[SUR_MAXL];   // sizes (outp: padded to 16)
    float *W[SUR_MAXL], *b[SUR_MAXL], *gW[SUR_MAXL], *gb[SUR_MAXL];
    float *mW[SUR_MAXL], *vW[SUR_MAXL], *mb[SUR_MAXL], *vb[SUR_MAXL];
    __nv_bfloat16 *W16[SUR_MAXL];    // [outp][in]  BF16 copy of W
    __nv_bfloat16 *WT16[SUR_MAXL];   // [in][outp]  BF16 copy of W^T
    int t;                       // Adam steps taken
    int bmax;                    // rows per forward/backward chunk (multiple of 128)
    __nv_bfloat16 *A[SUR_MAXL + 1];  // activations [bmax][in_l] (A[0] = features)
    __nv_bfloat16 *AT[SUR_MAXL + 1]; // the same transposed, [in_l][bmax]
    float *Z[SUR_MAXL];              // pre-activations [bmax][outp]
    __nv_bfloat16 *dZ[SUR_MAXL];     // loss gradients [bmax][outp]
    __nv_bfloat16 *dZT[SUR_MAXL];    // the same transposed, [outp][bmax]
    float *dZ32[SUR_MAXL];           // FP32 copy (bias gradients)
    float *wpart;                    // weight-gradient partials [split][outp][in]
    double *ms;                  // mu, sigma of log|M|^2 (device)
    double *part;                // loss partial sums
    float *y;                    // standardised targets of a chunk
    int *err;                    // device error word of the bounded waits
    uint32_t debug_extra_tx;     // test hook: extra bytes the GEMMs' operand barrier expects
    double *bpart;               // bias-gradient partials [bmax / 128][outp]
    int *dstate;                 // device training state (k_step_advance)
    double *dloss;               // device sum of batch losses of an epoch
    cudaStream_t cap;            // private stream the training step is captured on
};

namespace {

int sur_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? MG_ERR_NO_MEMORY : mg_cuda_fail(e); }

#define SCHECK(x)                                   \
    do {                                            \
        cudaError_t _e = (x);                       \
        if (_e != cudaSuccess) return sur_fail(_e); \
    } while (0)

void free_sur(mg_surrogate *s) {
    if (!s) return;
    for (int l = 0; l < SUR_MAXL; l++) {
        cudaFree(s->W[l]); cudaFree(s->b[l]); cudaFree(s->gW[l]); cudaFree(s->gb[l]);
        cudaFree(s->mW[l]); cudaFree(s->vW[l]); cudaFree(s->mb[l]); cudaFree(s->vb[l]);
        cudaFree(s->W16[l]); cudaFree(s->WT16[l]); cudaFree(s->Z[l]); cudaFree(s->dZ[l]);
        cudaFree(s->dZT[l]); cudaFree(s->dZ32[l]);
    }
    for (int l = 0; l <= SUR_MAXL; l++) {
        cudaFree(s->A[l]);
        cudaFree(s->AT[l]);
    }
    cudaFree(s->wpart); cudaFree(s->ms); cudaFree(s->part); cudaFree(s->y); cudaFree(s->err);
    cudaFree(s->dstate); cudaFree(s->dloss); cudaFree(s->bpart);
    if (s->cap) cudaStreamDestroy(s->cap);
    delete s;
}

int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

long long pad_rows(long long m) { return (m + MROWS - 1) / MROWS * MROWS; }

// column tile of a GEMM with N output columns (a multiple of 16)
int pick_nt(int N) {
    for (int nt = 64; nt >= 16; nt >>= 1)
        if (N % nt == 0) return nt;
    return 16;
}

// weight-gradient splits of a batch of M rows (64-row K chunks, 4 per split)
int wsplits(long long M) {
    const long long ch = M / 64;
    return (int)(ch % 4 == 0 ? ch / 4 : ch / 2);
}

// forward pass over rows [0, M) of s->A[0] (M a multiple of 128)
int forward(mg_surrogate *s, long long M, cudaStream_t st) {
    for (int l = 0; l < s->nl; l++) {
        const bool last = (l == s->nl - 1);
        mg_mlp_epi ep;
        memset(&ep, 0, sizeof(ep));
        ep.bias = s->b[l];
        ep.Z = s->Z[l];
        ep.A = last ? nullptr : s->A[l + 1];
        ep.AT = last ? nullptr : s->AT[l + 1];
        ep.ldz = s->outp[l];
        ep.ldt = s->bmax;
        ep.m_valid = (int)M;
        ep.n_valid = s->outp[l];
        SCHECK(mg_launch_mlp_gemm(last ? MG_MLP_FWD_OUT : MG_MLP_FWD, s->A[l], M, s->in[l], s->W16[l],
                                  s->outp[l], s->in[l], s->in[l], M, s->outp[l], pick_nt(s->outp[l]), 1,
                                  ep, s->err, st, s->debug_extra_tx));
    }
    return MG_OK;
}

// backward pass (needs forward + k_loss): fills gW, gb
int backward(mg_surrogate *s, long long M, cudaStream_t st) {
    const int ns = wsplits(M);
    for (int l = s->nl - 1; l >= 0; l--) {
        mg_mlp_epi ep;
        memset(&ep, 0, sizeof(ep));
        ep.part = s->wpart;
        ep.ldz = s->in[l];
        ep.m_valid = s->outp[l];
        ep.n_valid = s->in[l];
        // gW[n][k] = sum_m dZ[m][n] A[m][k]: X = dZ^T [outp][batch], Y = A^T [in][batch]
        SCHECK(mg_launch_mlp_gemm(MG_MLP_WGRAD, s->dZT[l], s->outp[l], s->bmax, s->AT[l], s->in[l],
                                  s->bmax, (int)M, pad_rows(s->outp[l]), s->in[l], pick_nt(s->in[l]), ns,
                                  ep, s->err, st, s->debug_extra_tx));
        const long long nw = (long long)s->outp[l] * s->in[l];
        const int nchunk = (int)((M + BIAS_ROWS - 1) / BIAS_ROWS);
        mg_note_launch();
        k_bias_part<<<dim3((unsigned)blocks_for(s->outp[l], 32), (unsigned)nchunk), 256, 0, st>>>(
            s->dZ32[l], M, s->outp[l], s->bpart);
        mg_note_launch();
        k_wgrad_reduce<<<blocks_for(nw, 256), 256, 0, st>>>(s->wpart, ns, nw, s->gW[l], s->bpart, nchunk,
                                                           s->outp[l], s->gb[l]);
        if (l > 0) {
            // dZ_l-1 = (dZ_l W_l) * silu'(Z_l-1): X = dZ_l [batch][outp], Y = W_l^T [in][outp]
            mg_mlp_epi ed;
            memset(&ed, 0, sizeof(ed));
            ed.Zprev = s->Z[l - 1];
            ed.dZ = s->dZ[l - 1];
            ed.dZT = s->dZT[l - 1];
            ed.dZ32 = s->dZ32[l - 1];
            ed.ldz = s->in[l];
            ed.ldt = s->bmax;
            ed.m_valid = (int)M;
            ed.n_valid = s->in[l];
            SCHECK(mg_launch_mlp_gemm(MG_MLP_BWD_DATA, s->dZ[l], M, s->outp[l], s->WT16[l], s->in[l],
                                      s->outp[l], s->outp[l], M, s->in[l], pick_nt(s->in[l]), 1, ed,
                                      s->err, st, s->debug_extra_tx));
        }
    }
    SCHECK(cudaGetLastError());
    return MG_OK;
}

// status of the bounded waits so far (synchronises the stream; clears it)
int device_status(mg_surrogate *s, cudaStream_t st) {
    int h = 0;
    SCHECK(cudaMemcpyAsync(&h, s->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCHECK(cudaStreamSynchronize(st));
    if (h) {
        SCHECK(cudaMemsetAsync(s->err, 0, sizeof(int), st));
        return MG_ERR_DEVICE_TIMEOUT;
    }
    return MG_OK;
}

// BF16 copies of W ([outp][in]) and W^T ([in][outp]) from FP32 host values
// (rows >= out zero)
int upload_w16(mg_surrogate *s, int l, const float *w) {
    const int ro = s->outp[l], ci = s->in[l];
    std::vector<__nv_bfloat16> w16((size_t)ro * ci), wt((size_t)ro * ci);
    for (int r = 0; r < ro; r++)
        for (int c = 0; c < ci; c++) {
            const __nv_bfloat16 v = __float2bfloat16_rn(r < s->out[l] ? w[(size_t)r * ci + c] : 0.0f);
            w16[(size_t)r * ci + c] = v;
            wt[(size_t)c * ro + r] = v;
        }
    SCHECK(cudaMemcpy(s->W16[l], w16.data(), w16.size() * 2, cudaMemcpyHostToDevice));
    SCHECK(cudaMemcpy(s->WT16[l], wt.data(), wt.size() * 2, cudaMemcpyHostToDevice));
    return MG_OK;
}

}  // namespace

extern "C" {

int mg_sur_create(int nin, int hidden, int nhidden, uint64_t seed, int bmax, mg_surrogate **out) {
    if (!out || nin < 1 || nin % 16 || hidden < 16 || hidden % 16 || nhidden < 1 ||
        nhidden + 1 > SUR_MAXL || bmax < 16 || bmax % 16)
        return MG_ERR_BAD_ARG;
    *out = nullptr;
    mg_surrogate *s = new mg_surrogate();
    memset(s, 0, sizeof(*s));
    s->nl = nhidden + 1;
    s->bmax = (int)pad_rows(bmax);
    bmax = s->bmax;
    int wmax = 0;
    for (int l = 0; l < s->nl; l++) {
        s->in[l] = (l == 0) ? nin : hidden;
        s->out[l] = (l == s->nl - 1) ? 1 : hidden;
        s->outp[l] = (s->out[l] + WM - 1) / WM * WM;
        if (s->outp[l] * s->in[l] > wmax) wmax = s->outp[l] * s->in[l];
    }
    // Glorot-uniform initial weights from a seeded generator (host), biases 0
    uint64_t st = seed * 6364136223846793005ULL + 1442695040888963407ULL;
    auto uni = [&]() {
        st = st * 6364136223846793005ULL + 1442695040888963407ULL;
        return ((st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    int rc = MG_OK;
    for (int l = 0; l < s->nl && rc == MG_OK; l++) {
        const size_t nw = (size_t)s->outp[l] * s->in[l], nb = s->outp[l];
        std::vector<float> w(nw, 0.0f);
        const double lim = sqrt(6.0 / (s->in[l] + s->out[l]));
        for (int r = 0; r < s->out[l]; r++)
            for (int c = 0; c < s->in[l]; c++) w[(size_t)r * s->in[l] + c] = (float)((2 * uni() - 1) * lim);
        cudaError_t e = cudaSuccess;
        float **f[] = {&s->W[l], &s->gW[l], &s->mW[l], &s->vW[l]};
        for (auto p : f)
            if (e == cudaSuccess && (e = cudaMalloc(p, nw * 4)) == cudaSuccess) e = cudaMemset(*p, 0, nw * 4);
        float **g[] = {&s->b[l], &s->gb[l], &s->mb[l], &s->vb[l]};
        for (auto p : g)
            if (e == cudaSuccess && (e = cudaMalloc(p, nb * 4)) == cudaSuccess) e = cudaMemset(*p, 0, nb * 4);
        if (e == cudaSuccess) e = cudaMalloc(&s->W16[l], nw * 2);
        if (e == cudaSuccess) e = cudaMalloc(&s->WT16[l], nw * 2);
        if (e == cudaSuccess) e = cudaMemcpy(s->W[l], w.data(), nw * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&s->Z[l], (size_t)bmax * s->outp[l] * 4);
        if (e == cudaSuccess) e = cudaMalloc(&s->dZ[l], (size_t)bmax * s->outp[l] * 2);
        if (e == cudaSuccess) e = cudaMalloc(&s->dZT[l], (size_t)bmax * s->outp[l] * 2);
        if (e == cudaSuccess) e = cudaMalloc(&s->dZ32[l], (size_t)bmax * s->outp[l] * 4);
        if (e == cudaSuccess) e = cudaMalloc(&s->A[l + 1], (size_t)bmax * s->outp[l] * 2);
        if (e == cudaSuccess) e = cudaMalloc(&s->AT[l + 1], (size_t)bmax * s->outp[l] * 2);
        if (e != cudaSuccess) rc = sur_fail(e);
        if (rc == MG_OK) rc = upload_w16(s, l, w.data());
    }
    if (rc == MG_OK) {
        cudaError_t e = cudaMalloc(&s->A[0], (size_t)bmax * nin * 2);
        if (e == cudaSuccess) e = cudaMalloc(&s->AT[0], (size_t)bmax * nin * 2);
        // at most bmax / 128 splits (2 chunks of 64 rows each) for any batch
        if (e == cudaSuccess) e = cudaMalloc(&s->wpart, (size_t)(bmax / 128) * wmax * 4);
        if (e == cudaSuccess) e = cudaMalloc(&s->ms, 2 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&s->part, (size_t)(bmax / 256 + 1) * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&s->y, (size_t)bmax * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&s->err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(s->err, 0, sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&s->dstate, 2 * sizeof(int));
        int omax = 0;
        for (int l = 0; l < s->nl; l++) omax = s->outp[l] > omax ? s->outp[l] : omax;
        if (e == cudaSuccess) e = cudaMalloc(&s->bpart, (size_t)(bmax / BIAS_ROWS) * omax * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&s->dloss, sizeof(double));
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
        const double ms0[2] = {0.0, 1.0};
        if (e == cudaSuccess) e = cudaMemcpy(s->ms, ms0, sizeof(ms0), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = sur_fail(e);
    }
    if (rc != MG_OK) {
        free_sur(s);
        return rc;
    }
    *out = s;
    return MG_OK;
}

void mg_sur_destroy(mg_surrogate *s) { free_sur(s); }

// parameters as FP32 [W_0 (out x in), b_0 (out), W_1, b_1, ...] (unpadded)
int mg_sur_param_count(const mg_surrogate *s, int64_t *n) {
    if (!s || !n) return MG_ERR_BAD_ARG;
    int64_t c = 0;
    for (int l = 0; l < s->nl; l++) c += (int64_t)s->out[l] * s->in[l] + s->out[l];
    *n = c;
    return MG_OK;
}

static int copy_params(mg_surrogate *s, float *host, int to_host, int grads) {
    size_t off = 0;
    for (int l = 0; l < s->nl; l++) {
        const size_t nw = (size_t)s->out[l] * s->in[l];
        float *W = grads ? s->gW[l] : s->W[l];
        float *b = grads ? s->gb[l] : s->b[l];
        cudaError_t e;
        if (to_host) {
            e = cudaMemcpy(host + off, W, nw * 4, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(host + off + nw, b, s->out[l] * 4, cudaMemcpyDeviceToHost);
        } else {
            e = cudaMemcpy(W, host + off, nw * 4, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(b, host + off + nw, s->out[l] * 4, cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return sur_fail(e);
        if (!to_host) {
            const int rc = upload_w16(s, l, host + off);
            if (rc) return rc;
        }
        off += nw + s->out[l];
    }
    return MG_OK;
}

int mg_sur_get_params(mg_surrogate *s, float *host) {
    if (!s || !host) return MG_ERR_BAD_ARG;
    return copy_params(s, host, 1, 0);
}
int mg_sur_set_params(mg_surrogate *s, const float *host) {
    if (!s || !host) return MG_ERR_BAD_ARG;
    return copy_params(s, const_cast<float *>(host), 0, 0);
}
int mg_sur_get_grads(mg_surrogate *s, float *host) {
    if (!s || !host) return MG_ERR_BAD_ARG;
    return copy_params(s, host, 1, 1);
}

// Copies an internal buffer of the last forward/backward pass to the host
// (FP32 out[rows][cols], padded widths): which = 0 activations A[layer]
// (layer 0 = features), 1 pre-activations Z[layer], 2 gradients dZ[layer] (FP32).
int mg_sur_debug_buffer(mg_surrogate *s, int which, int layer, int rows, float *out) {
    if (!s || !out || rows < 1 || rows > s->bmax || layer < 0) return MG_ERR_BAD_ARG;
    int cols = 0;
    if (which == 0 && layer <= s->nl - 1) {
        cols = layer == 0 ? s->in[0] : s->outp[layer - 1];
        std::vector<__nv_bfloat16> h((size_t)rows * cols);
        SCHECK(cudaMemcpy(h.data(), s->A[layer], h.size() * 2, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < h.size(); i++) out[i] = __bfloat162float(h[i]);
        return MG_OK;
    }
    if ((which == 1 || which == 2) && layer < s->nl) {
        cols = s->outp[layer];
        SCHECK(cudaMemcpy(out, which == 1 ? s->Z[layer] : s->dZ32[layer], (size_t)rows * cols * 4,
                          cudaMemcpyDeviceToHost));
        return MG_OK;
    }
    return MG_ERR_BAD_ARG;
}

// mu, sigma of log|M|^2 over me_dev[n]
int mg_sur_fit_target(mg_surrogate *s, const double *me, int64_t n, void *stream) {
    if (!s || !me || n < 2) return MG_ERR_BAD_ARG;
    mg_note_launch();
    k_logstats<<<1, 256, 0, (cudaStream_t)stream>>>(me, n, s->ms);
    SCHECK(cudaGetLastError());
    return MG_OK;
}

int mg_sur_get_target_stats(mg_surrogate *s, double *mu_sigma) {
    if (!s || !mu_sigma) return MG_ERR_BAD_ARG;
    SCHECK(cudaMemcpy(mu_sigma, s->ms, 2 * sizeof(double), cudaMemcpyDeviceToHost));
    return MG_OK;
}

// Loss and gradients for one batch (rows of momenta [m][npar][4] with
// targets y_dev[m] = standardised log|M|^2, FP32); m multiple of 16, <= bmax.
// The batch is padded to a multiple of 128 rows with zero features and zero
// loss gradient.
int mg_sur_loss_grad(mg_surrogate *s, const double *mom, int npar, const float *y, int m,
                     double *loss_out, void *stream) {
    if (!s || !mom || !y || m < 16 || m % 16 || m > s->bmax || npar < 2) return MG_ERR_BAD_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const long long M = pad_rows(m);
    mg_note_launch();
    k_features<<<blocks_for(M, 128), 128, 0, st>>>(mom, m, M, npar, s->in[0], s->A[0], s->AT[0], s->bmax);
    int rc = forward(s, M, st);
    if (rc) return rc;
    const int nb = blocks_for(M, 256);
    mg_note_launch();
    k_loss<<<nb, 256, 0, st>>>(s->Z[s->nl - 1], M, m, s->outp[s->nl - 1], y, s->dZ[s->nl - 1],
                               s->dZT[s->nl - 1], s->bmax, s->dZ32[s->nl - 1], s->part);
    rc = backward(s, M, st);
    if (rc) return rc;
    if (loss_out) {
        std::vector<double> h(nb);
        SCHECK(cudaMemcpyAsync(h.data(), s->part, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
        rc = device_status(s, st);
        if (rc) return rc;
        double t = 0.0;
        for (double v : h) t += v;
        *loss_out = t / m;
    }
    return MG_OK;
}

int mg_sur_adam(mg_surrogate *s, double lr, void *stream) {
    if (!s || !(lr > 0)) return MG_ERR_BAD_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    s->t++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)s->t), c2 = 1.0f - powf(b2, (float)s->t);
    for (int l = 0; l < s->nl; l++) {
        const long long nw = (long long)s->outp[l] * s->in[l];
        mg_note_launch();
        k_adam<<<blocks_for(nw, 256), 256, 0, st>>>(s->W[l], s->mW[l], s->vW[l], s->gW[l], s->W16[l],
                                                   s->WT16[l], s->outp[l], s->in[l], (float)lr, b1, b2,
                                                   1e-8f, c1, c2);
        mg_note_launch();
        k_adam<<<blocks_for(s->outp[l], 256), 256, 0, st>>>(s->b[l], s->mb[l], s->vb[l], s->gb[l], nullptr,
                                                           nullptr, 1, s->outp[l], (float)lr, b1, b2,
                                                           1e-8f, c1, c2);
    }
    SCHECK(cudaGetLastError());
    return MG_OK;
}

// One training step on batch dstate[0] of `batch` rows of mom / me (device-
// side batch index and Adam step count, so the same launches serve every
// step): targets, features, forward, loss (added to dloss), backward, Adam,
// advance of the device state.
static int train_step(mg_surrogate *s, const double *mom, int npar, const double *me, int batch,
                      double lr, cudaStream_t st) {
    const long long M = pad_rows(batch);
    mg_note_launch();
    k_target<<<blocks_for(batch, 256), 256, 0, st>>>(me, batch, s->ms, s->y, s->dstate);
    mg_note_launch();
    k_features<<<blocks_for(M, 128), 128, 0, st>>>(mom, batch, M, npar, s->in[0], s->A[0], s->AT[0], s->bmax,
                                                  s->dstate);
    int rc = forward(s, M, st);
    if (rc) return rc;
    const int nb = blocks_for(M, 256);
    mg_note_launch();
    k_loss<<<nb, 256, 0, st>>>(s->Z[s->nl - 1], M, batch, s->outp[s->nl - 1], s->y, s->dZ[s->nl - 1],
                               s->dZT[s->nl - 1], s->bmax, s->dZ32[s->nl - 1], s->part);
    mg_note_launch();
    k_loss_acc<<<1, 1, 0, st>>>(s->part, nb, s->dloss);
    rc = backward(s, M, st);
    if (rc) return rc;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int l = 0; l < s->nl; l++) {
        const long long nw = (long long)s->outp[l] * s->in[l];
        mg_note_launch();
        k_adam<<<blocks_for(nw, 256), 256, 0, st>>>(s->W[l], s->mW[l], s->vW[l], s->gW[l], s->W16[l],
                                                   s->WT16[l], s->outp[l], s->in[l], (float)lr, b1, b2,
                                                   1e-8f, 1.0f, 1.0f, s->dstate + 1);
        mg_note_launch();
        k_adam<<<blocks_for(s->outp[l], 256), 256, 0, st>>>(s->b[l], s->mb[l], s->vb[l], s->gb[l], nullptr,
                                                           nullptr, 1, s->outp[l], (float)lr, b1, b2,
                                                           1e-8f, 1.0f, 1.0f, s->dstate + 1);
    }
    mg_note_launch();
    k_step_advance<<<1, 1, 0, st>>>(s->dstate);
    SCHECK(cudaGetLastError());
    return MG_OK;
}

// Training: targets from me_dev (standardised with mg_sur_fit_target's mu,
// sigma), full batches in data order, `epochs` passes, Adam after each batch.
// The first step runs as plain launches; the step is then captured once as a
// CUDA graph (on the surrogate's private stream; it reads the batch index and
// the Adam step from device memory) and replayed for every later step on the
// caller's stream, so a step costs one graph launch instead of about thirty.
int mg_sur_train(mg_surrogate *s, const double *mom, int npar, const double *me, int64_t n,
                 int epochs, int batch, double lr, void *stream, double *last_epoch_loss) {
    if (!s || !mom || !me || batch < 16 || batch % 16 || batch > s->bmax || n < batch || epochs < 1 ||
        !(lr > 0))
        return MG_ERR_BAD_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nbatch = n / batch;
    int h0[2] = {0, s->t};   // pageable source: copied before the call returns
    SCHECK(cudaMemcpyAsync(s->dstate, h0, sizeof(h0), cudaMemcpyHostToDevice, st));
    SCHECK(cudaMemsetAsync(s->dloss, 0, sizeof(double), st));
    cudaGraphExec_t exec = nullptr;
    int rc = MG_OK;
    for (int ep = 0; ep < epochs && !rc; ep++) {
        cudaError_t e = cudaMemsetAsync(s->dstate, 0, sizeof(int), st);   // batch index 0
        if (e == cudaSuccess && ep == epochs - 1) e = cudaMemsetAsync(s->dloss, 0, sizeof(double), st);
        if (e != cudaSuccess) {
            rc = sur_fail(e);
            break;
        }
        for (int64_t bi = 0; bi < nbatch && !rc; bi++) {
            if (exec) {
                e = cudaGraphLaunch(exec, st);
                if (e != cudaSuccess) rc = sur_fail(e);
                continue;
            }
            rc = train_step(s, mom, npar, me, batch, lr, st);
            if (rc || ep * nbatch + bi + 1 == epochs * nbatch) continue;
            // capture the step once (nothing runs during capture)
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const int rs = train_step(s, mom, npar, me, batch, lr, s->cap);
                e = cudaStreamEndCapture(s->cap, &graph);
                if (rs) rc = rs;
            }
            if (!rc && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (!rc && e != cudaSuccess) rc = sur_fail(e);
        }
    }
    if (exec) cudaGraphExecDestroy(exec);
    double hloss = 0.0;
    if (!rc) {
        const cudaError_t e = cudaMemcpyAsync(&hloss, s->dloss, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = sur_fail(e);
    }
    if (!rc) rc = device_status(s, st);   // synchronises the stream
    if (rc) return rc;
    s->t += (int)(epochs * nbatch);
    if (last_epoch_loss) *last_epoch_loss = hloss / ((double)nbatch * batch);
    return MG_OK;
}

int mg_sur_debug_inject_stall(mg_surrogate *s, unsigned int extra_bytes) {
    if (!s) return MG_ERR_BAD_ARG;
    s->debug_extra_tx = extra_bytes;
    return MG_OK;
}

int mg_sur_device_status(mg_surrogate *s, void *stream) {
    if (!s) return MG_ERR_BAD_ARG;
    return device_status(s, (cudaStream_t)stream);
}

// Prediction of log|M|^2 for n events (chunks of bmax rows; n arbitrary).
int mg_sur_predict(mg_surrogate *s, const double *mom, int npar, int64_t n, double *logme,
                   void *stream) {
    if (!s || !mom || !logme || n < 0) return MG_ERR_BAD_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    for (int64_t e0 = 0; e0 < n; e0 += s->bmax) {
        const int64_t c = (n - e0 < s->bmax) ? n - e0 : s->bmax;
        const long long M = pad_rows(c);
        mg_note_launch();
        k_features<<<blocks_for(M, 128), 128, 0, st>>>(mom + e0 * npar * 4, c, M, npar, s->in[0], s->A[0],
                                                      s->AT[0], s->bmax);
        int rc = forward(s, M, st);
        if (rc) return rc;
        mg_note_launch();
        k_pred<<<blocks_for(c, 256), 256, 0, st>>>(s->Z[s->nl - 1], s->outp[s->nl - 1], c, s->ms, logme + e0);
    }
    SCHECK(cudaGetLastError());
    return MG_OK;
}

// Checkpoint: "MGSUR001", layer sizes, Adam step, mu/sigma, then per layer
// W, b, m_W, v_W, m_b, v_b (FP32, padded shapes).
int mg_sur_save(mg_surrogate *s, const char *path) {
    if (!s || !path) return MG_ERR_BAD_ARG;
    FILE *f = fopen(path, "wb");
    if (!f) return MG_ERR_BAD_ARG;
    int rc = MG_OK;
    double ms[2];
    int32_t hdr[2 + 2 * SUR_MAXL] = {s->nl, s->t};
    for (int l = 0; l < s->nl; l++) {
        hdr[2 + 2 * l] = s->in[l];
        hdr[3 + 2 * l] = s->out[l];
    }
    if (cudaMemcpy(ms, s->ms, sizeof(ms), cudaMemcpyDeviceToHost) != cudaSuccess) rc = MG_ERR_CUDA;
    if (!rc && (fwrite("MGSUR001", 1, 8, f) != 8 || fwrite(hdr, sizeof(hdr), 1, f) != 1 ||
                fwrite(ms, sizeof(ms), 1, f) != 1))
        rc = MG_ERR_BAD_ARG;
    for (int l = 0; l < s->nl && !rc; l++) {
        const size_t nw = (size_t)s->outp[l] * s->in[l], nb = s->outp[l];
        float *arr[] = {s->W[l], s->b[l], s->mW[l], s->vW[l], s->mb[l], s->vb[l]};
        size_t len[] = {nw, nb, nw, nw, nb, nb};
        for (int k = 0; k < 6 && !rc; k++) {
            std::vector<float> h(len[k]);
            if (cudaMemcpy(h.data(), arr[k], len[k] * 4, cudaMemcpyDeviceToHost) != cudaSuccess) rc = MG_ERR_CUDA;
            else if (fwrite(h.data(), 4, len[k], f) != len[k]) rc = MG_ERR_BAD_ARG;
        }
    }
    fclose(f);
    return rc;
}

int mg_sur_load(mg_surrogate *s, const char *path) {
    if (!s || !path) return MG_ERR_BAD_ARG;
    FILE *f = fopen(path, "rb");
    if (!f) return MG_ERR_BAD_ARG;
    char magic[8];
    int32_t hdr[2 + 2 * SUR_MAXL];
    double ms[2];
    int rc = MG_OK;
    if (fread(magic, 1, 8, f) != 8 || memcmp(magic, "MGSUR001", 8) || fread(hdr, sizeof(hdr), 1, f) != 1 ||
        fread(ms, sizeof(ms), 1, f) != 1 || hdr[0] != s->nl)
        rc = MG_ERR_BAD_ARG;
    for (int l = 0; l < s->nl && !rc; l++)
        if (hdr[2 + 2 * l] != s->in[l] || hdr[3 + 2 * l] != s->out[l]) rc = MG_ERR_BAD_ARG;
    for (int l = 0; l < s->nl && !rc; l++) {
        const size_t nw = (size_t)s->outp[l] * s->in[l], nb = s->outp[l];
        float *arr[] = {s->W[l], s->b[l], s->mW[l], s->vW[l], s->mb[l], s->vb[l]};
        size_t len[] = {nw, nb, nw, nw, nb, nb};
        for (int k = 0; k < 6 && !rc; k++) {
            std::vector<float> h(len[k]);
            if (fread(h.data(), 4, len[k], f) != len[k]) rc = MG_ERR_BAD_ARG;
            else if (cudaMemcpy(arr[k], h.data(), len[k] * 4, cudaMemcpyHostToDevice) != cudaSuccess) rc = MG_ERR_CUDA;
            if (!rc && k == 0) rc = upload_w16(s, l, h.data());
        }
    }
    if (!rc) {
        s->t = hdr[1];
        if (cudaMemcpy(s->ms, ms, sizeof(ms), cudaMemcpyHostToDevice) != cudaSuccess) rc = MG_ERR_CUDA;
    }
    fclose(f);
    return rc;
}

// Two-stage unweighting of n candidates (see the file header).  Inputs on
// the device: momenta [n][npar][4], phase-space weights phi[n], uniforms
// u1[n], u2[n].  Outputs (device): accept[n] (0/1), weight[n] (0 if
// rejected); *n_exact = candidates whose exact matrix element was computed.
// Workspace (what[n], flags, indices, gathered momenta and exact matrix
// elements of the stage-1 survivors) is allocated per call.
int mg_unweight2(mg_process *p, mg_surrogate *s, const double *mom, const double *phi,
                 const double *u1, const double *u2, int64_t n, double what_max, double r_max,
                 unsigned char *accept, double *weight, int64_t *n_exact, void *stream) {
    if (!p || !s || !mom || !phi || !u1 || !u2 || !accept || !weight || n < 1 || !(what_max > 0) ||
        !(r_max > 0))
        return MG_ERR_BAD_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int npar = p->tab->npar;
    const int nb = blocks_for(n, 1024);
    double *logme = nullptr, *what = nullptr, *mom1 = nullptr, *me1 = nullptr;
    unsigned char *flag = nullptr;
    int *bcount = nullptr;
    long long *idx = nullptr, *total = nullptr, htotal = 0;
    int rc = MG_OK;
    cudaError_t e = cudaMalloc(&logme, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&what, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&flag, n);
    if (e == cudaSuccess) e = cudaMalloc(&bcount, nb * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&total, sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&idx, n * sizeof(long long));
    if (e != cudaSuccess) rc = sur_fail(e);
    if (!rc) rc = mg_sur_predict(s, mom, npar, n, logme, st);
    if (!rc) {
        mg_note_launch();
        k_stage1<<<nb, 1024, 0, st>>>(logme, phi, u1, n, what_max, what, flag, bcount);
        mg_note_launch();
        k_scan<<<1, 32, 0, st>>>(bcount, nb, total);
        e = cudaMemcpyAsync(&htotal, total, sizeof(long long), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = sur_fail(e);
    }
    if (!rc && htotal > 0) {
        e = cudaMalloc(&mom1, htotal * npar * 4 * 8);
        if (e == cudaSuccess) e = cudaMalloc(&me1, htotal * 8);
        if (e != cudaSuccess) rc = sur_fail(e);
        if (!rc) {
            mg_note_launch();
            k_compact<<<nb, 1024, 0, st>>>(flag, bcount, n, mom, npar, idx, mom1);
            rc = mg_sigmakin(p, mom1, htotal, me1, st);
        }
    }
    if (!rc) {
        e = cudaMemsetAsync(accept, 0, n, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(weight, 0, n * 8, st);
        if (e != cudaSuccess) rc = sur_fail(e);
        if (!rc && htotal > 0) {
            mg_note_launch();
            k_stage2<<<blocks_for(htotal, 256), 256, 0, st>>>(idx, me1, htotal, phi, what, u2, what_max,
                                                             r_max, accept, weight);
        }
        e = cudaStreamSynchronize(st);
        if (!rc && e != cudaSuccess) rc = sur_fail(e);
    }
    if (!rc) rc = device_status(s, st);   // a bounded wait of the surrogate's GEMMs gave up
    cudaFree(logme); cudaFree(what); cudaFree(flag); cudaFree(bcount); cudaFree(total);
    cudaFree(idx); cudaFree(mom1); cudaFree(me1);
    if (!rc && n_exact) *n_exact = htotal;
    return rc;
}

}  // extern "C"
