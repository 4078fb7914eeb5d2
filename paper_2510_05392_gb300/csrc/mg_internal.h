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
    int nops, nscat;
    long long denom;         // colour-matrix common denominator D
    double iden;             // averaging factor
    double flops_diagram;    // algorithmic FP64 flops per helicity (diagrams)
    double flops_colour;     // algorithmic FP64 flops per helicity (colour sum)
    const int32_t *ops;      // [nops][8]
    const int32_t *scat;     // [nscat]
    const int32_t *chat;     // [ncolor][ncolor], D * C
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

#ifdef __cplusplus
#include <cuda_runtime.h>
// Launchers (mg_kernels.cu).  All asynchronous on `stream`.
// units: work units (gluon-helicity configuration << 4 | mask of the good
// (top, antitop) helicity combinations, bit 2*bt + btb), nunits of them.
cudaError_t mg_launch_sigmakin(const mg_dev_proc &dp, const double *mom, int64_t nevt,
                               const int *units, int nunits, int tpe, int block, double *me,
                               double *me_hel, cudaStream_t stream);
cudaError_t mg_launch_helmask(const double *me_hel, int64_t n, int nhel, double rel,
                              unsigned char *mask, cudaStream_t stream);
#endif
