/*
 * mgpu -- leading-order QCD matrix elements for g g -> t t~ + n g on one
 * NVIDIA GB300 (sm_103a).  C ABI.
 *
 * What the library computes is the per-event matrix element engine of the
 * paper (Sec. 2.2, "sigmaKin": input 4*npar doubles per event, output one
 * matrix element per event): external wavefunctions, internal wavefunctions
 * and amplitudes of every Feynman diagram, accumulated into colour-flow
 * amplitudes ("jamps"), contracted with the colour matrix (Sec. 3.3, Eq. "jcj":
 * J^H C J = A^T C A + B^T C B with J = A + iB), summed over the good
 * helicities (Sec. 2.2 and Sec. 4.6, helicity filtering) and averaged over
 * initial spins/colours and identical final gluons.
 *
 * Conventions
 *   particle order   g1 g2 t t~ g5 ... g_npar (g1 along +z, g2 along -z)
 *   momenta          (E, px, py, pz) in GeV, float64, layout [nevt][npar][4]
 *                    contiguous, 8-byte aligned, in device memory on the
 *                    process's device
 *   output           float64 [nevt] in device memory, GeV^(4-2*npar)
 *   helicity index   h in [0, 2^npar): bit (npar-1-i) set <=> particle i has
 *                    positive helicity
 *   streams          every compute call is asynchronous and ordered on the
 *                    given cudaStream_t (NULL = legacy default stream).
 *                    Every evaluation path keeps per-process workspaces
 *                    grown on demand (FP64: the jamp buffer, 64 * ncolor
 *                    bytes per diagram-kernel thread, at most 24 GiB: a
 *                    larger call runs as several launches, and the jamps stay
 *                    in local memory when it cannot be allocated; the
 *                    mixed precision path, the table-file process and the
 *                    extras: their own buffers as well): the first call, and
 *                    any call with more events than before, allocates
 *                    (cudaFree/cudaMalloc, which can synchronise the
 *                    device); later calls of at most that size do not (so
 *                    before capturing calls in a CUDA graph, make one call
 *                    of at least the captured size outside the capture).
 *                    mg_filter_helicities_noalloc never allocates.
 *                    Calls on one process share its workspaces, so they must
 *                    not overlap on the GPU: issue them on one stream (or
 *                    order the streams), or use one process per stream.
 *
 * Ownership: the caller owns all momentum/output buffers.  The library owns
 * the opaque process handle, its device tables and its workspaces, all
 * released by mg_process_destroy.
 *
 * Errors: every function returns MG_OK (0) or a negative status; nothing
 * aborts, exits or traps.  mg_status_string() names a status.
 */
#ifndef MGPU_H
#define MGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MG_OK = 0,
    MG_ERR_BAD_PROCESS = -1,   /* unknown or unsupported process string      */
    MG_ERR_BAD_ARG = -2,       /* null/misaligned/host pointer, bad size/flag */
    MG_ERR_NOT_FILTERED = -3,  /* mg_sigmakin before mg_filter_helicities     */
    MG_ERR_CUDA = -4,          /* a CUDA runtime call failed                  */
    MG_ERR_DEVICE_TIMEOUT = -5,/* a bounded device-side wait gave up          */
    MG_ERR_NO_MEMORY = -6,     /* device allocation failed                    */
    MG_ERR_UNSUPPORTED = -7    /* feature not available for this process     */
};

enum { MG_HEL_FILTERED = 0, MG_HEL_ALL = 1 };
enum { MG_FP64 = 0, MG_MIXED_BF16 = 1 };

typedef struct mg_process mg_process; /* opaque, library-owned */

typedef struct {
    double mt;       /* top mass [GeV]                                      */
    double wt;       /* top width [GeV], used in every top propagator        */
    double alphas;   /* fixed strong coupling, g_s = sqrt(4 pi alphas)      */
    int hel_mode;    /* MG_HEL_FILTERED (filter first) or MG_HEL_ALL        */
    int precision;   /* MG_FP64 (all FP64) or MG_MIXED_BF16 (FP64 diagrams, */
                     /* colour sum on tcgen05 tensor cores: jamps split in  */
                     /* three BF16 pieces, D*C in two, FP32 accumulation,   */
                     /* FP64 epilogue; above 128 flows over the block upper */
                     /* triangle in 128-colour blocks with FP64 block sums; */
                     /* mg_sigmakin_hel is then MG_ERR_UNSUPPORTED)        */
} mg_params;

typedef struct {
    int npar;             /* external particles                          */
    int ngluon;           /* gluons, incoming included                   */
    int ndiagrams;        /* Feynman diagrams (4-gluon vertex counted once) */
    int nterms;           /* diagram terms (each 4-gluon vertex has 3)   */
    int ncolor;           /* colour flows                                 */
    int nhel;             /* 2^npar helicity combinations                 */
    int ngood;            /* good helicities (-1 before filtering)        */
    int nslot;            /* gluon-wavefunction slots per thread (1 variant) */
    int nslot_top;        /* top-line slots per thread (2 helicity variants) */
    int nops;             /* wavefunction/amplitude operations            */
    int njamp_updates;    /* jamp updates per helicity                    */
    int64_t denom;        /* colour-matrix common denominator D           */
    double iden;          /* averaging factor                             */
    double flops_diagram; /* algorithmic FP64 flops per helicity: diagrams */
    double flops_colour;  /* algorithmic FP64 flops per helicity: colour sum */
    int nchannel;         /* single-diagram-enhancement channels          */
} mg_info;

/* Create a process from its description, e.g. "g g > t t~ g g".  Supported:
 * g g > t t~ followed by 0..4 final gluons (5 final gluons: the table-file
 * entry point below).  Uploads the process tables to
 * the current CUDA device.  params may be NULL (mt 173, wt 1.4915,
 * alphas 0.118, filtered helicities, FP64). */
int mg_process_create(const char *process, const mg_params *params, mg_process **out);

/* Create g g > t t~ g g g g g (2 -> 7: 5040 colour flows; the paper could
 * build it for CPUs only, Table "ggtt5g") from the binary table file the
 * process compiler writes (compiler/emit.py emit_blob: "MGPROC02" header,
 * program, jamp scatter, colour row by relative ordering, flow orderings,
 * channel colour factors).
 * Every index of the program is checked against its pools before anything
 * reaches the device; a damaged or foreign file gives MG_ERR_BAD_PROCESS.
 * Runs with its wavefunction state in HBM (about 1.9 MB per thread, three
 * 128-thread blocks per SM while half the free memory holds them) and an
 * FP64 colour sum over the block upper triangle of the 5040 x 5040 colour
 * matrix (built on the device, 203 MB); with MG_MIXED_BF16 the colour sum
 * runs on the tensor cores instead (jamps as three BF16 pieces, D*C as
 * C_hi + C_lo, FP32 accumulation per 128-colour block, blocks added in FP64;
 * relative error about 1e-6).  mg_sigmakin, mg_sigmakin_hel, mg_filter_helicities,
 * mg_color_matrix, mg_sigmakin_ex (in both precisions) and the timing hooks
 * work as for the other processes; the batch calls and
 * mg_filter_helicities_noalloc return MG_ERR_UNSUPPORTED. */
int mg_process_create_from_tables(const char *table_path, const mg_params *params, mg_process **out);

/* Helicity filter (Sec. 2.2 and Sec. 4.6 of the paper: keep the helicities with
 * a non-zero contribution).  Evaluates all 2^npar helicities in parallel on
 * the n test events momenta_dev[n][npar][4] and keeps h when
 * |M_h|^2 > 1e-14 * max_h' |M_h'|^2 on any of them.  Synchronises the stream
 * (initialisation step).  n in [1, 65536].  *ngood_out may be NULL. */
int mg_filter_helicities(mg_process *p, const double *momenta_dev, int64_t n, void *stream,
                         int *ngood_out);

/* Same rule and result as mg_filter_helicities, without allocating device
 * memory.  The paper has no counterpart; it exists for callers that cannot
 * call cudaMalloc/cudaFree: code whose device memory is owned by another
 * allocator (a framework's caching allocator, a fixed memory budget), and
 * code that must not trigger the device-wide synchronisation of cudaFree
 * while other streams run.  Its scratch is a fixed 128.25 KiB array inside the
 * library (held on every GPU that loads it until exit), so n is limited to
 * 1..64 test events (larger n: MG_ERR_BAD_ARG).  The first call on a device
 * looks up the array's device address (make it before any stream capture);
 * the current device must be the process's device.  All calls share the
 * array: calls whose work overlaps on the GPU (other threads, other streams)
 * race and must be serialised by the caller.  Its uploads of the helicity
 * list are ordered on `stream` (none goes through the legacy default
 * stream); like every call on a process it must not overlap that process's
 * other work on the GPU.  Synchronises the stream. */
int mg_filter_helicities_noalloc(mg_process *p, const double *momenta_dev, int64_t n, void *stream,
                                 int *ngood_out);

/* Matrix elements of nevt events: me_out_dev[nevt] (float64, device).
 * nevt = 0 is a no-op (the pointers are then not inspected and may be
 * NULL).  Asynchronous on stream.  Requires a prior
 * mg_filter_helicities unless hel_mode == MG_HEL_ALL.  Non-finite momenta
 * give non-finite results (not checked). */
int mg_sigmakin(mg_process *p, const double *momenta_dev, int64_t nevt, double *me_out_dev,
                void *stream);

/* Per-helicity contributions: me_hel_dev[nevt][2^npar] (float64, device),
 * already averaged (their sum over h is the matrix element); helicities that
 * are not good are written as 0.  me_out_dev may be NULL. */
int mg_sigmakin_hel(mg_process *p, const double *momenta_dev, int64_t nevt, double *me_out_dev,
                    double *me_hel_dev, void *stream);

/* Status of the device-side work issued so far for p on stream: synchronises
 * the stream, returns MG_ERR_DEVICE_TIMEOUT (and clears it) when a bounded
 * wait inside a kernel gave up since the last call (the kernel then wrote no
 * valid result for the affected events), MG_ERR_CUDA on a CUDA error, else
 * MG_OK. */
int mg_device_status(mg_process *p, void *stream);

/* Per-event extras of sigmaKin (FP64 path, and both precisions of the
 * table-file process; all pointers device, optional unless stated).  The paper's production kernel also takes an event-by-
 * event alpha_s, random numbers for a helicity and a colour choice, and a
 * channel id for single-diagram enhancement (Sec. 2.2):
 *   alphas_dev       [nevt] per-event alpha_s.  Every vertex is QCD, so
 *                    |M|^2 scales as alpha_s^ngluon: the matrix element is
 *                    rescaled by (alphas[e] / params.alphas)^ngluon.
 *   channel          single-diagram-enhancement channel of every event, or
 *                    -1.  The channels are the diagrams that MadEvent's
 *                    single diagram enhancement uses (table "complexity",
 *                    row 3 of the paper): the Feynman diagrams made of
 *                    three-point vertices only, 3 / 15 / 105 / 945 for 2 to
 *                    5 gluons (10395 and 135135 for 6 and 7).  Channel c is
 *                    the c-th in the order of mg_sde_channels.
 *   channel_ids_dev  [nevt] int32, per-event channels (the paper's
 *                    event-by-event channel identifier); overrides channel
 *                    when not NULL.  An id outside [0, nchannel) gives a
 *                    weight of 0 for that event.
 *   sde_weight_dev   out [nevt] (required with a channel or channel ids):
 *                    sum_h |D_c,h|^2 / sum_h sum_c' |D_c',h|^2 over the good
 *                    helicities h and the channels c', D_c,h the amplitude of
 *                    diagram c alone (its colour coefficients have modulus
 *                    one); diagrams with a four-gluon vertex enter neither
 *                    sum
 *   flow_weight_dev  out [nevt][ncolor]: sum over good helicities of |J_s|^2
 *                    (jamps without couplings)
 *   rnd_hel_dev, hel_out_dev   uniforms in [0,1) and out [nevt] helicity index:
 *                    first h whose running sum of |M_h|^2 exceeds r * sum
 *   rnd_col_dev, col_out_dev   likewise for the colour flow with weights
 *                    flow_weight (h and flow choices need their uniforms)
 * me_out_dev may be NULL.  Uses cached per-process workspaces (grown on
 * demand). */
typedef struct {
    const double *alphas_dev;
    int channel;
    double *sde_weight_dev;
    double *flow_weight_dev;
    const double *rnd_hel_dev;
    int *hel_out_dev;
    const double *rnd_col_dev;
    int *col_out_dev;
    const int *channel_ids_dev;
} mg_sigmakin_extras;
int mg_sigmakin_ex(mg_process *p, const double *momenta_dev, int64_t nevt,
                   const mg_sigmakin_extras *extras, double *me_out_dev, void *stream);

/* Launch shape: threads per event (1..32, power of two) and threads per
 * block (multiple of 32, <= 128: the diagram kernel keeps three 128-thread
 * blocks resident per SM).  0 keeps the current value. */
int mg_set_launch(mg_process *p, int threads_per_event, int block);

int mg_process_info(const mg_process *p, mg_info *out);

/* Integer colour matrix D*C (row-major ncolor x ncolor) and D, exactly as
 * the colour sum uses them.  Flow s is the string t^{a_s1}..t^{a_sn} with
 * orderings in lexicographic permutation order of the gluons (g1 g2 g5 ...). */
int mg_color_matrix(const mg_process *p, int64_t *ints_out, int64_t *denom_out);

/* Good-helicity mask [2^npar] (1 = good) after filtering (or all ones in
 * MG_HEL_ALL mode).  MG_ERR_NOT_FILTERED before. */
int mg_helicity_mask(const mg_process *p, uint8_t *mask_out);

/* Single-diagram-enhancement channels (the diagrams MadEvent's single
 * diagram enhancement uses, table "complexity" row 3 and Sec. 2.2 of the
 * paper: the Feynman diagrams made of three-point vertices only).  A channel
 * is identified by its diagram's colour factor in the flow basis of
 * mg_color_matrix: codes_out[c][s] (int8, [nchannel][ncolor], may be NULL)
 * is 0 when flow s is absent, else the coefficient divided by the channel's
 * first one (in flow order) coded 1: +1, 2: -1, 3: +i, 4: -i.  Channels are
 * numbered in the lexicographic order of these code rows.  *nchannel_out
 * (may be NULL) receives the count.  Host-side; nothing runs on the GPU. */
int mg_sde_channels(const mg_process *p, int *nchannel_out, int8_t *codes_out);

void mg_process_destroy(mg_process *p);

/* ---- uneven multi-process batches in one persistent launch -------------
 * Blocks of events of several FP64 processes (each filtered, <= 5 gluons)
 * evaluated by one persistent kernel: warps take 32-slot chunks (slot =
 * event x thread of that event) from an atomic counter, heaviest process
 * first.  The paper has no batch API; it runs one process per application
 * (Sec. 2.3) and replays repeated launches as CUDA graphs (Sec. 4.1).
 *
 * mg_batch_create records the blocks (device pointers momenta[i]
 * [nevt[i]][npar_i][4] and me_out[i] [nevt[i]], owned by the caller and read
 * on every run), allocates the jamp buffers of the persistent kernel's
 * threads (64 x the largest colour-flow count bytes per thread, about 0.45
 * GB on a GB300 when a 5-gluon process is in the batch) and copies each
 * process's current helicity list (a later
 * mg_filter_helicities of a process does not change the batch); the batch
 * reads its processes' device tables on every run, so it must be destroyed
 * before any of them; mg_batch_run replays the launch as a CUDA graph (captured on
 * the first run on a private stream, asynchronous on `stream` afterwards);
 * mg_batch_autotune times the batch for several threads-per-event choices of
 * every block and CTAs per SM (coordinate descent, `reps` launches each,
 * synchronous) and keeps the fastest, writing its time to *best_ms_out;
 * mg_batch_config reports the choice (tpe_out[nproc], in the caller's
 * order).  mg_sigmakin_batch is the one-shot form (create, one launch,
 * synchronise, destroy). */
typedef struct mg_batch mg_batch;
int mg_batch_create(int nproc, mg_process *const *procs, const double *const *momenta_dev,
                    const int64_t *nevt, double *const *me_out_dev, mg_batch **out);
int mg_batch_run(mg_batch *b, void *stream);
int mg_batch_autotune(mg_batch *b, void *stream, int reps, double *best_ms_out);
int mg_batch_config(const mg_batch *b, int *tpe_out, int *ctas_per_sm_out);
void mg_batch_destroy(mg_batch *b);
int mg_sigmakin_batch(int nproc, mg_process *const *procs, const double *const *momenta_dev,
                      const int64_t *nevt, double *const *me_out_dev, void *stream);

const char *mg_status_string(int status);

/* Last CUDA error string seen by the library on this thread ("" if none). */
const char *mg_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif
