// The process handle behind the opaque mg_process of include/mgpu.h (shared
// by the host runtime files).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "mg_internal.h"

struct mg_process {
    const mg_proc_table *tab;
    int table_index;
    mg_params par;
    int device;
    int32_t *d_ops;
    int32_t *d_scat;
    double *d_cup;
    int *d_units;        // work units (device): gluon config << 4 | top-helicity mask
    int nunits;
    int ngood;           // -1 until filtered
    uint8_t mask[512];
    int tpe, block;      // launch shape
    double factor;
    // mixed precision: tensor-core colour sum (precision == MG_MIXED_BF16)
    int kp, np;                  // padded colour counts (K per piece, N)
    __nv_bfloat16 *d_cmat;       // [2*np][kp] BF16, D*C = hi + lo
    __nv_bfloat16 *d_jbuf;       // jamp rows of one chunk, [rows][3*kp] BF16
    long long jbuf_rows;
    int jbuf_nunits;             // unit count the buffer's padding was zeroed for
    double *d_part;              // partial colour sums of one chunk
    long long part_len;
    double2 *d_jg;               // jamps of every thread of a diagram launch
    size_t jg_bytes;
    int jg_off;                  // test hook: 1 = jamps updated in local memory
    size_t jg_max;               // test hook: buffer limit in bytes (0: the default)
    int *d_err;                  // device error word of the bounded waits
    uint32_t debug_extra_tx;     // test hook: extra bytes the TMA barrier expects
    // per-event extras (mg_sigmakin_ex): cached workspaces
    double *d_sel_hel;           // [cap][2^npar] per-helicity |M_h|^2
    double *d_sel_jw;            // [cap][ncolor] helicity-summed |J_s|^2
    long long sel_cap;
    // kernel timing (measurement hook): CUDA event pairs around each launch
    int timing;                  // 1 while enabled
    cudaEvent_t *tev;            // [2 * tcap]
    int *tkind;                  // [tcap] MG_KT_* of each recorded launch
    int tcap, tn, tdropped;
    // processes loaded from a table file, run with their state in HBM (mg_big.cu)
    int big;
    mg_proc_table *own_tab;      // host tables owned by the process
    long long *d_crow;           // device [ncolor] D*C by relative ordering
    signed char *d_cperm;        // device [ncolor][ngluon] flow orderings
    double *d_cbig;              // device [np][np] block upper triangle of D*C, k-major
    int big_np;                  // colours padded to the 64-colour tile
    double2 *d_scratch;          // per-thread wavefunction state, slot-major
    long long scratch_threads;   // threads the scratch holds
    long long big_threads;       // threads per launch (0: default)
    double *d_jrow;              // FP64 jamp rows of one chunk, colour-major
    long long jrow_items;        // items (padded) the row buffer holds
    double *d_qpart;             // per-tile colour sums of one chunk
    long long qpart_len;
    double *d_sde_item;          // per-item channel sums of one chunk (extras)
    long long sde_item_cap;      // items it holds
    void *d_kin;                 // kinematic tables of the events of one chunk
    long long kin_cap;           // events they hold
};

// kinds of timed launches
enum { MG_KT_DIAGRAM = 0, MG_KT_COLOUR = 1, MG_KT_EVENT_SUM = 2, MG_KT_NKIND = 3 };

// Timing of one launch: mg_timer_begin records the start event (returns the
// slot, or -1 when timing is off or the pool is full), mg_timer_end the stop.
int mg_timer_begin(mg_process *p, cudaStream_t s, int kind);
void mg_timer_end(mg_process *p, cudaStream_t s, int slot);

// helpers of mg_api.cu used by the other host files
int mg_check_dev_ptr(const void *ptr, int device);
int mg_cuda_fail(cudaError_t e);
mg_dev_proc mg_dev_view(const mg_process *p);
