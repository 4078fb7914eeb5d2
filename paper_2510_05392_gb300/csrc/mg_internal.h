// Internal declarations shared by the host runtime and the kernels.
#pragma once
#include <stdint.h>

#include "mgpu.h"

#ifdef __cplusplus
extern "C" {
#endif

// One compiled process: tables written by the process compiler
// (paper_2510_05392_gb300/compiler/emit.py).
typedef struct {
    const char *name;        // "ggttgg"
    const char *process;     // "g g > t t~ g g"
    int ngluon, npar, ndiagrams, nterms, ncolor;
    int nslot;               // gluon-wavefunction slots (one variant)
    int nslot_top;           // top-line slots (two helicity variants)
    int nslot_acc;           // amplitude accumulators of colour-factor groups
    int nops, nscat;
    long long denom;         // colour-matrix common denominator D
    double iden;             // averaging factor
    double flops_diagram;    // algorithmic FP64 flops per helicity (diagrams)
    double flops_colour;     // algorithmic FP64 flops per helicity (colour sum)
    const int32_t *ops;      // [nops][8]
    const int32_t *scat;     // [nscat]
    const int32_t *chat;     // [ncolor][ncolor], D * C (NULL for table-file processes)
    const int64_t *crow;     // table-file processes: D * C by relative ordering [ncolor]
    const int8_t *cperm;     // table-file processes: flow orderings [ncolor][ngluon]
    int nchannel;            // single-diagram-enhancement channels
    const int32_t *chan_off; // [nchannel + 1] offsets into chan_flows
    const int32_t *chan_flows; // per channel its colour factor: flow * 8 + code
} mg_proc_table;

const mg_proc_table *mg_tables(int *count);

#ifdef __cplusplus
}
#endif

// Opcodes of the wavefunction/amplitude program (compiler/program.py).
enum {
    MG_OP_EXT_G = 1,
    MG_OP_EXT_UB = 2,
    MG_OP_EXT_V = 3,
    MG_OP_V3 = 4,
    MG_OP_V4 = 5,
    MG_OP_FPRE = 6,
    MG_OP_FSUF = 7,
    MG_OP_XROW = 8,
    MG_OP_YCOL = 9,
    MG_OP_BIL = 10,
    MG_OP_AMP_SS = 11,
    MG_OP_AMP_VV = 12
};

// Device-side view of a process used by the launchers.
typedef struct {
    int table_index;                 // selects the kernel instantiation
    const int32_t *ops;              // device [nops][8]
    int nops;
    const int32_t *scat;             // device [nscat]
    const double *cup;               // device packed upper triangle of D*C, off-diagonals doubled
    int ncolor;
    double mt, wt;
    double factor;                   // g^(2n) / (iden * D)
} mg_dev_proc;

#define MG_TC_ERR_TIMEOUT 1   // device error word: a bounded wait ran out

// Optional per-event extras of the FP64 diagram kernel.
typedef struct {
    const double *alphas;  // per-event alpha_s [nevt] or NULL
    double alphas0;        // alpha_s the couplings were built with
    int channel;           // single-diagram-enhancement channel of every event, or -1
    const int *channel_ids;// per-event channels [nevt] (overrides channel) or NULL
    double *sde;           // out [nevt]: |D_channel|^2 / sum_channels |D|^2, or NULL
    double *jw;            // out [nevt][ncolor]: helicity-summed |J_s|^2, or NULL
} mg_extras;

// One process block of a multi-process batch (device copy read by the
// persistent kernel).  Slots [slot_begin, slot_end) are event * tpe + thread,
// padded to a multiple of 32 so that every warp works on one item.
typedef struct {
    const int32_t *ops;
    const int32_t *scat;
    const double *cup;
    const int *units;
    const double *mom;
    double *me;
    long long nevt;
    long long slot_begin, slot_end;
    double mt, wt, factor;
    int nops, nunits, tpe, table_index;
} mg_batch_item;

#ifdef __cplusplus
#include <cuda_bf16.h>
#include <cuda_runtime.h>
// Launchers (mg_kernels.cu, mg_colorsum_tc.cu).  All asynchronous on `stream`.
// units: work units (gluon-helicity configuration << 4 | mask of the good
// (top, antitop) helicity combinations, bit 2*bt + btb), nunits of them.
// jout != NULL: write the jamps as tensor-core GEMM rows (no FP64 colour sum,
// me/me_hel unused); row index ((e * nunits_pad + unit) * 4 + v) * 2 + re/im.
// jg != NULL: the jamps accumulate there through L2 reductions, jamp (c, v) of
// thread t at jg[(4 c + v) * T + t] with T = the launch's threads
// (ceil(nevt * tpe / block) * block), so jg holds 4 * ncolor * T double2;
// NULL: they stay in local memory.
cudaError_t mg_launch_sigmakin(const mg_dev_proc &dp, const double *mom, int64_t nevt,
                               const int *units, int nunits, int tpe, int block, double *me,
                               double *me_hel, cudaStream_t stream, __nv_bfloat16 *jout = nullptr,
                               int kp = 0, int nunits_pad = 0, const mg_extras *extras = nullptr,
                               double2 *jg = nullptr);
cudaError_t mg_launch_select(const double *me_hel, int nhel, const double *jw, int ncolor,
                             long long nevt, const double *rh, const double *rc, int *hel_out,
                             int *col_out, cudaStream_t stream);
cudaError_t mg_launch_helmask(const double *me_hel, int64_t n, int nhel, double rel,
                              unsigned char *mask, cudaStream_t stream);
// tensor-core colour sum over ncols_alloc (multiple of 128) GEMM rows of jbuf
// ([ncols][3*kp] BF16) with cmat ([2*np][kp] BF16: D*C split hi/lo), cpe
// rows per event (a power of two >= 8); writes mg_tc_parts_per_tile(cpe)
// partial sums per 128-row tile, mg_tc_parts_per_event(cpe) per event,
// contiguous per event
cudaError_t mg_launch_colorsum_tc(const __nv_bfloat16 *jbuf, long long ncols_alloc, int kp,
                                  const __nv_bfloat16 *cmat, int np, int ncolor, int cpe,
                                  uint32_t extra_tx, double *part, int *err, cudaStream_t stream);
cudaError_t mg_launch_event_sum(const double *part, long long nevt, int per_event, double factor,
                                double *me, cudaStream_t stream);
size_t mg_tc_smem_bytes(int kp, int np);
// processes with their state in HBM (mg_big.cu)
int mg_big_ngluon();
int mg_big_block();
int mg_big_blocks_per_sm(int *out);
size_t mg_big_state_bytes(int nslot, int nslot_top, int nslot_acc);
size_t mg_big_kin_bytes();   // kinematic tables of one event
cudaError_t mg_launch_build_cbig(const long long *row, const signed char *perm, int nc, int np,
                                 double *cbT, cudaStream_t stream);
cudaError_t mg_launch_sigmakin_big(const mg_dev_proc &dp, const double *mom, long long nitem,
                                   const int *units, int nunits, int nsg, int nsf, double2 *scratch,
                                   long long T, double *jrow, long long R, long long nipad,
                                   void *kin, cudaStream_t stream, int channel = -1,
                                   const int *channel_ids = nullptr, double *sde_item = nullptr);
cudaError_t mg_launch_flow_weights_big(const double *jrow, long long R, long long nipad,
                                       const int *units, int nunits, long long nevt, int ncolor,
                                       double *jw, cudaStream_t stream);
cudaError_t mg_launch_build_cmat_bf16(const long long *row, const signed char *perm, int nc, int kp,
                                     __nv_bfloat16 *cm, cudaStream_t stream);
cudaError_t mg_launch_rows_to_bf16(const double *jrow, long long R, int nsrc, int kp,
                                   __nv_bfloat16 *jb, cudaStream_t stream);
cudaError_t mg_launch_colour_big(const double *jrow, long long R, const double *cbT, int np,
                                 double *qpart, cudaStream_t stream);
cudaError_t mg_launch_event_sum_big(const double *qpart, long long R, int ntile, long long nipad,
                                    const int *units, int nunits, long long nevt, double factor,
                                    double *me, double *me_hel, cudaStream_t stream,
                                    const double *alphas = nullptr, double alphas0 = 0.0,
                                    const double *sde_item = nullptr, double *sde = nullptr);
// counts a kernel launch of the library (measurement; replays of captured
// graphs are not launches of this kind and are not counted)
void mg_note_launch();
int mg_tc_parts_per_tile(int cpe);
// tensor-core colour sum of the table-file process over the block upper
// triangle: jb [R][3*kp] BF16 rows, cmat [2*np][kp] (np == kp, multiples of
// 128); writes part[(2 I + half) * R + r] for the 2 np / 128 colour halves
cudaError_t mg_launch_rows_split(const double *rows, long long nrows, int nc, int kp,
                                 __nv_bfloat16 *jb, cudaStream_t stream);
cudaError_t mg_launch_event_sum_rows(const double *part, long long R, int ncols, int cpe, long long nevt,
                                     double factor, double *me, cudaStream_t stream);
cudaError_t mg_launch_colorsum_tc_big(const __nv_bfloat16 *jb, long long R, int kp,
                                      const __nv_bfloat16 *cmat, int np, uint32_t extra_tx,
                                      double *part, int *err, cudaStream_t stream);
int mg_tc_parts_per_event(int cpe);
// persistent multi-process kernel: counter reset + one launch of grid CTAs of
// 128 threads; jg (may be NULL): the threads' jamp buffers, 4 * (largest
// ncolor) * grid * 128 double2
cudaError_t mg_launch_batch(const mg_batch_item *d_items, int nitems, unsigned long long *d_counter,
                            long long total_slots, int grid, cudaStream_t stream,
                            double2 *jg = nullptr);
int mg_batch_ctas_per_sm(int *out);
int mg_sigmakin_occupancy(int table_index, int block, int *ctas_per_sm);
#define MG_BATCH_MAX_NGLUON 5   // processes the persistent kernel carries
#endif
