// Host runtime behind the C ABI declared in include/mgpu.h: process
// registry (compiled-in tables and table files), device tables, argument
// checks, helicity filtering, and the launch sequences of the FP64, mixed
// and HBM-state (2 -> 7) paths with their per-event extras.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>

#include "mg_internal.h"
#include "mgpu.h"

#include "mg_process.h"

namespace {

thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e) {
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return MG_ERR_CUDA;
}

#define MG_CUDA(call)                          \
    do {                                       \
        cudaError_t _e = (call);               \
        if (_e != cudaSuccess) return cuda_fail(_e); \
    } while (0)

std::string normalise(const char *s) {
    std::string out;
    bool sp = true;
    for (const char *c = s; *c; c++) {
        if (*c == ' ' || *c == '\t' || *c == '\n') {
            if (!sp) out.push_back(' ');
            sp = true;
        } else {
            out.push_back(*c);
            sp = false;
        }
    }
    while (!out.empty() && out.back() == ' ') out.pop_back();
    return out;
}

// A device pointer usable by this process: non-null, aligned (8 bytes unless
// stated), device (or managed) memory of the process's device.
int check_dev_ptr(const void *ptr, int device, int align = 8) {
    if (!ptr) return MG_ERR_BAD_ARG;
    if (reinterpret_cast<uintptr_t>(ptr) % align) return MG_ERR_BAD_ARG;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MG_ERR_BAD_ARG;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return MG_ERR_BAD_ARG;
    if (at.type == cudaMemoryTypeDevice && at.device != device) return MG_ERR_BAD_ARG;
    return MG_OK;
}

mg_dev_proc dev_view(const mg_process *p) {
    mg_dev_proc d;
    d.table_index = p->table_index;
    d.ops = p->d_ops;
    d.nops = p->tab->nops;
    d.scat = p->d_scat;
    d.cup = p->d_cup;
    d.ncolor = p->tab->ncolor;
    d.mt = p->par.mt;
    d.wt = p->par.wt;
    d.factor = p->factor;
    return d;
}

void free_proc(mg_process *p) {
    if (!p) return;
    cudaFree(p->d_ops);
    cudaFree(p->d_scat);
    cudaFree(p->d_cup);
    cudaFree(p->d_units);
    cudaFree(p->d_cmat);
    cudaFree(p->d_jbuf);
    cudaFree(p->d_part);
    cudaFree(p->d_err);
    cudaFree(p->d_sel_hel);
    cudaFree(p->d_sel_jw);
    for (int i = 0; i < 2 * p->tcap; i++) cudaEventDestroy(p->tev[i]);
    free(p->tev);
    free(p->tkind);
    cudaFree(p->d_crow);
    cudaFree(p->d_cperm);
    cudaFree(p->d_cbig);
    cudaFree(p->d_scratch);
    cudaFree(p->d_jrow);
    cudaFree(p->d_qpart);
    cudaFree(p->d_sde_item);
    cudaFree(p->d_kin);
    cudaFree(p->d_jg);
    if (p->own_tab) {
        free((void *)p->own_tab->ops);
        free((void *)p->own_tab->scat);
        free((void *)p->own_tab->crow);
        free((void *)p->own_tab->cperm);
        free((void *)p->own_tab->chan_off);
        free((void *)p->own_tab->chan_flows);
        free(p->own_tab);
    }
    free(p);
}

// Good-helicity mask -> work units: one per gluon-helicity configuration g
// that has a good helicity, with the 4-bit mask of its good (top, antitop)
// combinations (bit 2*bt + btb).  The upload is a plain cudaMemcpy, or, with
// async, a cudaMemcpyAsync ordered on stream s.
int set_hel_list(mg_process *p, const uint8_t *mask, bool async = false, cudaStream_t s = nullptr) {
    const int npar = p->tab->npar, ng = p->tab->ngluon;
    int units[128];
    int nu = 0, ngood = 0;
    for (int h = 0; h < (1 << npar); h++) p->mask[h] = mask[h] ? 1 : 0;
    for (int g = 0; g < (1 << ng); g++) {
        int m = 0;
        for (int v = 0; v < 4; v++) {
            int h = ((v >> 1) << (npar - 1 - 2)) | ((v & 1) << (npar - 1 - 3));
            for (int j = 0; j < ng; j++) {
                const int ip = (j < 2) ? j : j + 2;
                h |= ((g >> j) & 1) << (npar - 1 - ip);
            }
            if (mask[h]) {
                m |= 1 << v;
                ngood++;
            }
        }
        if (m) units[nu++] = (g << 4) | m;
    }
    if (nu > 0 && async)
        MG_CUDA(cudaMemcpyAsync(p->d_units, units, sizeof(int) * nu, cudaMemcpyHostToDevice, s));
    else if (nu > 0)
        MG_CUDA(cudaMemcpy(p->d_units, units, sizeof(int) * nu, cudaMemcpyHostToDevice));
    p->nunits = nu;
    p->ngood = ngood;
    return MG_OK;
}

// Tensor-core colour sum set-up: padded sizes and the BF16 colour matrix
// D*C = C_hi + C_lo (both parts exact in BF16; checked).
int setup_mixed(mg_process *p) {
    const mg_proc_table *t = p->tab;
    const int nc = t->ncolor;
    if (nc <= 128) {   // one tile holds every colour flow (32-colour rows up to 32 flows)
        p->kp = nc <= 32 ? 32 : 64 * ((nc + 63) / 64);
        p->np = 16 * ((nc + 15) / 16);
    } else {           // block upper triangle in 128-colour blocks
        p->kp = 128 * ((nc + 127) / 128);
        p->np = p->kp;
    }
    const size_t n = (size_t)2 * p->np * p->kp;
    __nv_bfloat16 *h = (__nv_bfloat16 *)calloc(n, sizeof(__nv_bfloat16));
    if (!h) return MG_ERR_NO_MEMORY;
    for (int i = 0; i < nc; i++)
        for (int j = 0; j < nc; j++) {
            const double c = (double)t->chat[i * nc + j];
            const __nv_bfloat16 hi = __float2bfloat16_rn((float)c);
            const double rem = c - (double)__bfloat162float(hi);
            const __nv_bfloat16 lo = __float2bfloat16_rn((float)rem);
            if ((double)__bfloat162float(hi) + (double)__bfloat162float(lo) != c) {
                free(h);
                return MG_ERR_UNSUPPORTED;
            }
            h[(size_t)i * p->kp + j] = hi;
            h[(size_t)(p->np + i) * p->kp + j] = lo;
        }
    cudaError_t e = cudaMalloc(&p->d_cmat, n * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_cmat, h, n * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice);
    free(h);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? MG_ERR_NO_MEMORY : cuda_fail(e);
    return MG_OK;
}

// ---------------------------------------------------------------------------
// Processes loaded from a table file and run with their state in HBM
// (mg_big.cu): chunks of events whose FP64 jamp rows fit 24 GiB; per chunk
// the rows are cleared, the diagram kernel accumulates the jamps into them,
// the colour-sum kernel forms every row's quadratic form per 64-colour tile
// and the event sum adds them up.
// Per-event extras of a table-file process (mg_sigmakin_ex): alphas [nevt]
// or NULL, channel (or per-event channel_ids) and sde [nevt] (NULL: no
// weights), flow weights jw [nevt][ncolor] or NULL.
struct BigExtras {
    const double *alphas;
    int channel;
    const int *channel_ids;
    double *sde;
    double *jw;
};

int sigmakin_big(mg_process *p, const double *mom, int64_t nevt, double *me, double *me_hel,
                 cudaStream_t s, const BigExtras *bx = nullptr) {
    const mg_proc_table *t = p->tab;
    const int nu = p->nunits;
    const int nhel = 1 << t->npar;
    if (nevt <= 0) return MG_OK;
    if (nu == 0) {
        if (me) MG_CUDA(cudaMemsetAsync(me, 0, sizeof(double) * nevt, s));
        return MG_OK;
    }
    const long long np = p->big_np;
    const bool mixed = p->par.precision == MG_MIXED_BF16;
    // FP64: one partial per 64-colour tile; mixed: per half of a 128-colour tile
    const int ntile = mixed ? 2 * p->kp / 128 : (int)(np / 64);
    const int ipad = mixed ? 16 : 8;   // items per padding unit: rows in whole 128-row tiles
    const long long row_limit = (24LL << 30) / (np * 8);      // rows of 24 GiB
    long long ev_chunk = row_limit / (8LL * nu);
    if (ev_chunk < 1) ev_chunk = 1;
    if (ev_chunk > nevt) ev_chunk = nevt;
    const long long nipad_max = (ev_chunk * nu + ipad - 1) / ipad * ipad;
    // threads: the resident blocks of every SM while the device has room for
    // their state, never more than the items of a chunk
    int nsm = 0, occ = 0;
    MG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device));
    if (mg_big_blocks_per_sm(&occ) != 0 || occ < 1) return MG_ERR_CUDA;
    const int blk = mg_big_block();
    const size_t state = mg_big_state_bytes(t->nslot, t->nslot_top, t->nslot_acc);
    long long T = p->big_threads;
    if (T <= 0) {
        size_t freeb = 0, totalb = 0;
        MG_CUDA(cudaMemGetInfo(&freeb, &totalb));
        const long long have = p->scratch_threads;
        T = (long long)occ * nsm * blk;
        while (T > blk && T > have && (size_t)(T - have) * state > freeb / 2) T -= blk;
    }
    // every thread holds one item (seconds of work) at a time: spread the
    // items of a full chunk evenly over whole waves of threads
    const long long waves = (ev_chunk * nu + T - 1) / T;
    T = ((ev_chunk * nu + waves - 1) / waves + blk - 1) / blk * blk;
    if (T > p->scratch_threads) {
        cudaFree(p->d_scratch);
        p->d_scratch = nullptr;
        p->scratch_threads = 0;
        cudaError_t e = cudaMalloc(&p->d_scratch, (size_t)T * state);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? MG_ERR_NO_MEMORY : cuda_fail(e);
        p->scratch_threads = T;
    }
    if (nipad_max > p->jrow_items) {
        cudaFree(p->d_jrow);
        cudaFree(p->d_qpart);
        p->d_jrow = nullptr;
        p->d_qpart = nullptr;
        p->jrow_items = 0;
        cudaError_t e = cudaMalloc(&p->d_jrow, sizeof(double) * np * 8 * nipad_max);
        if (e == cudaSuccess) e = cudaMalloc(&p->d_qpart, sizeof(double) * ntile * 8 * nipad_max);
        if (e == cudaSuccess && mixed) {
            cudaFree(p->d_jbuf);
            p->d_jbuf = nullptr;
            e = cudaMalloc(&p->d_jbuf, sizeof(__nv_bfloat16) * 3 * p->kp * 8 * nipad_max);
        }
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? MG_ERR_NO_MEMORY : cuda_fail(e);
        p->jrow_items = nipad_max;
    }
    const bool want_sde = bx && bx->sde;
    if (want_sde && nipad_max > p->sde_item_cap) {   // per-item channel sums, one chunk
        cudaFree(p->d_sde_item);
        p->d_sde_item = nullptr;
        p->sde_item_cap = 0;
        cudaError_t e = cudaMalloc(&p->d_sde_item, sizeof(double) * 8 * nipad_max);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? MG_ERR_NO_MEMORY : cuda_fail(e);
        p->sde_item_cap = nipad_max;
    }
    if (ev_chunk > p->kin_cap) {
        cudaFree(p->d_kin);
        p->d_kin = nullptr;
        p->kin_cap = 0;
        cudaError_t e = cudaMalloc(&p->d_kin, mg_big_kin_bytes() * (size_t)ev_chunk);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? MG_ERR_NO_MEMORY : cuda_fail(e);
        p->kin_cap = ev_chunk;
    }
    double *sde_item = want_sde ? p->d_sde_item : nullptr;
    int rc = MG_OK;
    const mg_dev_proc dp = dev_view(p);
    for (long long e0 = 0; e0 < nevt; e0 += ev_chunk) {
        const long long n = (nevt - e0 < ev_chunk) ? nevt - e0 : ev_chunk;
        const long long nitem = n * nu;
        const long long nip = (nitem + ipad - 1) / ipad * ipad;
        const long long R = 8 * nip;
        cudaError_t e = cudaMemsetAsync(p->d_jrow, 0, sizeof(double) * np * R, s);
        int slot = mg_timer_begin(p, s, MG_KT_DIAGRAM);
        if (e == cudaSuccess)
            e = mg_launch_sigmakin_big(dp, mom + e0 * t->npar * 4, nitem, p->d_units, nu, t->nslot,
                                       t->nslot_top, p->d_scratch, T, p->d_jrow, R, nip, p->d_kin, s,
                                       want_sde ? bx->channel : -1,
                                       want_sde && bx->channel_ids ? bx->channel_ids + e0 : nullptr,
                                       sde_item);
        mg_timer_end(p, s, slot);
        slot = mg_timer_begin(p, s, MG_KT_COLOUR);
        if (e == cudaSuccess && mixed) {
            e = mg_launch_rows_to_bf16(p->d_jrow, R, (int)np, p->kp, p->d_jbuf, s);
            if (e == cudaSuccess)
                e = mg_launch_colorsum_tc_big(p->d_jbuf, R, p->kp, p->d_cmat, p->np, p->debug_extra_tx,
                                              p->d_qpart, p->d_err, s);
        } else if (e == cudaSuccess) {
            e = mg_launch_colour_big(p->d_jrow, R, p->d_cbig, (int)np, p->d_qpart, s);
        }
        mg_timer_end(p, s, slot);
        slot = mg_timer_begin(p, s, MG_KT_EVENT_SUM);
        if (e == cudaSuccess)
            e = mg_launch_event_sum_big(p->d_qpart, R, ntile, nip, p->d_units, nu, n, p->factor,
                                        me ? me + e0 : nullptr, me_hel ? me_hel + e0 * nhel : nullptr, s,
                                        bx && bx->alphas ? bx->alphas + e0 : nullptr, p->par.alphas,
                                        sde_item, want_sde ? bx->sde + e0 : nullptr);
        mg_timer_end(p, s, slot);
        if (e == cudaSuccess && bx && bx->jw)
            e = mg_launch_flow_weights_big(p->d_jrow, R, nip, p->d_units, nu, n, t->ncolor,
                                           bx->jw + e0 * t->ncolor, s);
        if (e != cudaSuccess) {
            rc = cuda_fail(e);
            break;
        }
    }
    return rc;
}

// Checks every index a table-file program can use against its pools, so a
// damaged file is rejected on the host instead of addressing out of bounds.
bool valid_program(const mg_proc_table *t) {
    const int ng = t->ngluon, nsub = 1 << ng;
    const int nsg = t->nslot, nsf = t->nslot_top, nsa = t->nslot_acc;
    auto in = [](int x, int n) { return x >= 0 && x < n; };
    for (int i = 0; i < t->nops; i++) {
        const int32_t *r = t->ops + 8 * i;
        const int c = r[0], ay = r[1], az = r[2], aw = r[3], bx = r[4], by = r[5], bz = r[6], bw = r[7];
        bool ok;
        switch (c) {
            case MG_OP_EXT_G: ok = in(ay, nsg) && in(az, t->npar) && az != 2 && az != 3; break;
            case MG_OP_EXT_UB:
            case MG_OP_EXT_V: ok = in(ay, nsf); break;
            case MG_OP_V3: ok = in(ay, nsg) && in(az, nsg) && in(aw, nsg) && in(bx, nsub) && in(by, nsub); break;
            case MG_OP_V4:
                ok = in(ay, nsg) && in(az, nsg) && in(aw, nsg) && in(bx, nsg) && in(by, nsg) &&
                     in(bz, nsg) && in(bw, nsub);
                break;
            case MG_OP_FPRE:
            case MG_OP_FSUF: ok = in(ay, nsf) && in(az, nsf) && in(aw, nsg) && in(bx, nsub); break;
            case MG_OP_XROW: ok = in(ay, nsf) && in(az, nsf) && in(aw, nsg); break;
            case MG_OP_YCOL: ok = in(ay, nsf) && in(az, nsg) && in(aw, nsf); break;
            case MG_OP_BIL: ok = in(az, nsf) && in(aw, nsf); break;
            case MG_OP_AMP_SS:
            case MG_OP_AMP_VV:
                ok = (c == MG_OP_AMP_SS ? in(az, nsf) && in(aw, nsf) : in(aw, nsg)) && bx >= 0 &&
                     by >= 0 && (long long)bx + by <= t->nscat && (bz == -1 || in(bz, nsa)) &&
                     (ay == -1 || in(ay, t->nchannel));
                break;
            default: ok = false;
        }
        if (!ok) return false;
    }
    for (int i = 0; i < t->nscat; i++)
        if (t->scat[i] < 0 || (t->scat[i] >> 2) >= t->ncolor) return false;
    if (t->chan_off[0] != 0) return false;
    for (int c = 0; c < t->nchannel; c++) {
        if (t->chan_off[c + 1] <= t->chan_off[c]) return false;
        for (int i = t->chan_off[c]; i < t->chan_off[c + 1]; i++) {
            const int f = t->chan_flows[i];
            if (f < 0 || (f >> 3) >= t->ncolor || (f & 7) < 1 || (f & 7) > 4) return false;
        }
    }
    for (int a = 0; a < t->ncolor; a++) {
        unsigned seen = 0;
        for (int q = 0; q < ng; q++) {
            const int x = t->cperm[a * ng + q];
            if (x < 0 || x >= ng || ((seen >> x) & 1u)) return false;
            seen |= 1u << x;
        }
    }
    return true;
}

mg_proc_table *read_table_file(const char *path, int *status) {
    *status = MG_ERR_BAD_PROCESS;
    FILE *f = fopen(path, "rb");
    if (!f) return nullptr;
    char magic[8];
    int32_t h[13];
    int64_t den;
    double dv[3];
    mg_proc_table *t = (mg_proc_table *)calloc(1, sizeof(mg_proc_table));
    bool ok = t && fread(magic, 1, 8, f) == 8 && memcmp(magic, "MGPROC02", 8) == 0 &&
              fread(h, sizeof(int32_t), 13, f) == 13 && fread(&den, 8, 1, f) == 1 &&
              fread(dv, 8, 3, f) == 3;
    if (ok) {
        ok = h[0] == 2 && h[1] == mg_big_ngluon() && h[2] == h[1] + 2 && h[3] > 0 && h[4] > 0 &&
             h[5] >= 0 && h[6] > 0 && h[7] > 0 && h[8] > 0 && h[12] > 0 && den > 0;
        long long fact = 1;
        for (int i = 2; i <= h[1]; i++) fact *= i;
        ok = ok && h[3] == fact;
    }
    if (ok) {
        t->ngluon = h[1];
        t->npar = h[2];
        t->ncolor = h[3];
        t->nops = h[4];
        t->nscat = h[5];
        t->nslot = h[6];
        t->nslot_top = h[7];
        t->nslot_acc = h[8];
        t->ndiagrams = h[10];
        t->nterms = h[11];
        t->nchannel = h[12];
        t->denom = den;
        t->iden = dv[0];
        t->flops_diagram = dv[1];
        t->flops_colour = dv[2];
        int32_t *ops = (int32_t *)malloc(sizeof(int32_t) * 8 * (size_t)t->nops);
        int32_t *scat = (int32_t *)malloc(sizeof(int32_t) * (t->nscat > 0 ? t->nscat : 1));
        int64_t *row = (int64_t *)malloc(sizeof(int64_t) * t->ncolor);
        int8_t *perm = (int8_t *)malloc((size_t)t->ncolor * t->ngluon);
        int32_t *choff = (int32_t *)malloc(sizeof(int32_t) * ((size_t)t->nchannel + 1));
        t->ops = ops;
        t->scat = scat;
        t->crow = row;
        t->cperm = perm;
        t->chan_off = choff;
        ok = ops && scat && row && perm && choff &&
             fread(ops, sizeof(int32_t), 8 * (size_t)t->nops, f) == 8 * (size_t)t->nops &&
             fread(scat, sizeof(int32_t), t->nscat, f) == (size_t)t->nscat &&
             fread(row, sizeof(int64_t), t->ncolor, f) == (size_t)t->ncolor &&
             fread(perm, 1, (size_t)t->ncolor * t->ngluon, f) == (size_t)t->ncolor * t->ngluon &&
             fread(choff, sizeof(int32_t), (size_t)t->nchannel + 1, f) == (size_t)t->nchannel + 1;
        // each channel has at most 2^(ngluon - 1) flows (one per planar ordering)
        ok = ok && choff[t->nchannel] > 0 && choff[t->nchannel] <= t->nchannel * (1 << (t->ngluon - 1));
        if (ok) {
            int32_t *chf = (int32_t *)malloc(sizeof(int32_t) * (size_t)choff[t->nchannel]);
            t->chan_flows = chf;
            ok = chf && fread(chf, sizeof(int32_t), choff[t->nchannel], f) == (size_t)choff[t->nchannel] &&
                 fgetc(f) == EOF && valid_program(t);
        }
    }
    fclose(f);
    if (!ok) {
        if (t) {
            free((void *)t->ops);
            free((void *)t->scat);
            free((void *)t->crow);
            free((void *)t->cperm);
            free((void *)t->chan_off);
            free((void *)t->chan_flows);
            free(t);
        }
        return nullptr;
    }
    t->name = "ggttggggg";
    t->process = "g g > t t~ g g g g g";
    *status = MG_OK;
    return t;
}

int pow2_at_least(int x) {
    int v = 1;
    while (v < x) v <<= 1;
    return v;
}

int default_tpe(int npar) {
    // threads per event (each thread takes 2^ngluon / tpe work units of
    // four helicities): enough threads for small batches of the small
    // processes, few redundant per-event kinematics for the large ones
    // (measured on GB300 with the jamp buffer: ggtt best at 2, ggttgg flat
    // from 1 to 4, ggttggg 8 and 16 equal, ggttgggg 32 3.6% faster than 16
    // on 16,384 events)
    switch (npar) {
        case 4: return 2;
        case 5: return 2;
        case 6: return 4;
        case 7: return 8;
        case 8: return 32;
        default: return 16;
    }
}

}  // namespace

extern "C" {

const char *mg_status_string(int s) {
    switch (s) {
        case MG_OK: return "ok";
        case MG_ERR_BAD_PROCESS: return "unknown or unsupported process";
        case MG_ERR_BAD_ARG: return "bad argument";
        case MG_ERR_NOT_FILTERED: return "helicities not filtered";
        case MG_ERR_CUDA: return "CUDA error";
        case MG_ERR_DEVICE_TIMEOUT: return "device wait timed out";
        case MG_ERR_NO_MEMORY: return "out of device memory";
        case MG_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

const char *mg_last_cuda_error(void) { return g_cuda_err; }

int mg_process_create(const char *process, const mg_params *params, mg_process **out) {
    if (!process || !out) return MG_ERR_BAD_ARG;
    *out = nullptr;
    mg_params par = {173.0, 1.4915, 0.118, MG_HEL_FILTERED, MG_FP64};
    if (params) par = *params;
    if (!(par.mt > 0.0) || !(par.wt >= 0.0) || !(par.alphas > 0.0)) return MG_ERR_BAD_ARG;
    if (par.hel_mode != MG_HEL_FILTERED && par.hel_mode != MG_HEL_ALL) return MG_ERR_BAD_ARG;
    if (par.precision != MG_FP64 && par.precision != MG_MIXED_BF16) return MG_ERR_BAD_ARG;
    int ntab = 0;
    const mg_proc_table *tabs = mg_tables(&ntab);
    const std::string want = normalise(process);
    int idx = -1;
    for (int i = 0; i < ntab; i++)
        if (want == tabs[i].process) idx = i;
    if (idx < 0) return MG_ERR_BAD_PROCESS;
    const mg_proc_table *t = &tabs[idx];

    mg_process *p = (mg_process *)calloc(1, sizeof(mg_process));
    if (!p) return MG_ERR_NO_MEMORY;
    p->tab = t;
    p->table_index = idx;
    p->par = par;
    p->ngood = -1;
    p->tpe = default_tpe(t->npar);
    p->block = 128;
    const double gs = sqrt(4.0 * M_PI * par.alphas);
    p->factor = pow(gs, 2 * t->ngluon) / (t->iden * (double)t->denom);
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        free_proc(p);
        return cuda_fail(e);
    }
    // packed upper triangle of D*C with doubled off-diagonals (exact in FP64)
    const int nc = t->ncolor;
    const size_t ntri = (size_t)nc * (nc + 1) / 2;
    double *cup = (double *)malloc(sizeof(double) * ntri);
    if (!cup) {
        free_proc(p);
        return MG_ERR_NO_MEMORY;
    }
    size_t w = 0;
    for (int i = 0; i < nc; i++)
        for (int j = i; j < nc; j++) cup[w++] = (i == j ? 1.0 : 2.0) * (double)t->chat[i * nc + j];
    int st = MG_OK;
#define TRY(call)                                   \
    do {                                            \
        cudaError_t _e = (call);                    \
        if (_e != cudaSuccess) {                    \
            st = (_e == cudaErrorMemoryAllocation) ? MG_ERR_NO_MEMORY : cuda_fail(_e); \
            goto fail;                              \
        }                                           \
    } while (0)
    TRY(cudaMalloc(&p->d_ops, sizeof(int32_t) * 8 * t->nops));
    TRY(cudaMalloc(&p->d_scat, sizeof(int32_t) * (t->nscat > 0 ? t->nscat : 1)));
    TRY(cudaMalloc(&p->d_cup, sizeof(double) * ntri));
    TRY(cudaMalloc(&p->d_units, sizeof(int) * 128));
    TRY(cudaMemcpy(p->d_ops, t->ops, sizeof(int32_t) * 8 * t->nops, cudaMemcpyHostToDevice));
    if (t->nscat > 0)
        TRY(cudaMemcpy(p->d_scat, t->scat, sizeof(int32_t) * t->nscat, cudaMemcpyHostToDevice));
    TRY(cudaMemcpy(p->d_cup, cup, sizeof(double) * ntri, cudaMemcpyHostToDevice));
    TRY(cudaMalloc(&p->d_err, sizeof(int)));
    TRY(cudaMemset(p->d_err, 0, sizeof(int)));
    if (par.precision == MG_MIXED_BF16) {
        st = setup_mixed(p);
        if (st != MG_OK) goto fail;
    }
#undef TRY
    free(cup);
    if (par.hel_mode == MG_HEL_ALL) {
        uint8_t all[512];
        memset(all, 1, sizeof(all));
        st = set_hel_list(p, all);
        if (st != MG_OK) {
            free_proc(p);
            return st;
        }
    }
    *out = p;
    return MG_OK;
fail:
    free(cup);
    free_proc(p);
    return st;
}

int mg_process_create_from_tables(const char *path, const mg_params *params, mg_process **out) {
    if (!path || !out) return MG_ERR_BAD_ARG;
    *out = nullptr;
    mg_params par = {173.0, 1.4915, 0.118, MG_HEL_FILTERED, MG_FP64};
    if (params) par = *params;
    if (!(par.mt > 0.0) || !(par.wt >= 0.0) || !(par.alphas > 0.0)) return MG_ERR_BAD_ARG;
    if (par.hel_mode != MG_HEL_FILTERED && par.hel_mode != MG_HEL_ALL) return MG_ERR_BAD_ARG;
    if (par.precision != MG_FP64 && par.precision != MG_MIXED_BF16) return MG_ERR_BAD_ARG;
    int st = MG_OK;
    mg_proc_table *t = read_table_file(path, &st);
    if (!t) return st;
    if (par.precision == MG_MIXED_BF16)   // D*C = C_hi + C_lo must be exact in BF16
        for (int i = 0; i < t->ncolor; i++) {
            const float c = (float)t->crow[i];
            const __nv_bfloat16 hi = __float2bfloat16_rn(c);
            const __nv_bfloat16 lo = __float2bfloat16_rn(c - __bfloat162float(hi));
            if ((double)__bfloat162float(hi) + (double)__bfloat162float(lo) != (double)t->crow[i]) {
                free((void *)t->ops);
                free((void *)t->scat);
                free((void *)t->crow);
                free((void *)t->cperm);
                free(t);
                return MG_ERR_UNSUPPORTED;
            }
        }
    mg_process *p = (mg_process *)calloc(1, sizeof(mg_process));
    if (!p) {
        free((void *)t->ops);
        free((void *)t->scat);
        free((void *)t->crow);
        free((void *)t->cperm);
        free(t);
        return MG_ERR_NO_MEMORY;
    }
    p->own_tab = t;
    p->tab = t;
    p->big = 1;
    p->table_index = -1;
    p->par = par;
    p->ngood = -1;
    p->tpe = 1;
    p->block = mg_big_block();
    const double gs = sqrt(4.0 * M_PI * par.alphas);
    p->factor = pow(gs, 2 * t->ngluon) / (t->iden * (double)t->denom);
    p->big_np = 64 * ((t->ncolor + 63) / 64);
    const size_t np = (size_t)p->big_np;
    const bool mixed = par.precision == MG_MIXED_BF16;
    p->kp = mixed ? 128 * ((t->ncolor + 127) / 128) : 0;
    p->np = p->kp;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_ops, sizeof(int32_t) * 8 * t->nops);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_scat, sizeof(int32_t) * (t->nscat > 0 ? t->nscat : 1));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_units, sizeof(int) * 128);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_crow, sizeof(long long) * t->ncolor);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_cperm, (size_t)t->ncolor * t->ngluon);
    if (e == cudaSuccess && !mixed) e = cudaMalloc(&p->d_cbig, sizeof(double) * np * np);
    if (e == cudaSuccess && mixed)
        e = cudaMalloc(&p->d_cmat, sizeof(__nv_bfloat16) * 2 * (size_t)p->kp * p->kp);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_ops, t->ops, sizeof(int32_t) * 8 * t->nops, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && t->nscat > 0)
        e = cudaMemcpy(p->d_scat, t->scat, sizeof(int32_t) * t->nscat, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_crow, t->crow, sizeof(long long) * t->ncolor, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_cperm, t->cperm, (size_t)t->ncolor * t->ngluon, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !mixed)
        e = mg_launch_build_cbig(p->d_crow, p->d_cperm, t->ncolor, (int)np, p->d_cbig, 0);
    if (e == cudaSuccess && mixed)
        e = mg_launch_build_cmat_bf16(p->d_crow, p->d_cperm, t->ncolor, p->kp, p->d_cmat, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_proc(p);
        return e == cudaErrorMemoryAllocation ? MG_ERR_NO_MEMORY : cuda_fail(e);
    }
    if (par.hel_mode == MG_HEL_ALL) {
        uint8_t all[512];
        memset(all, 1, sizeof(all));
        st = set_hel_list(p, all);
        if (st != MG_OK) {
            free_proc(p);
            return st;
        }
    }
    *out = p;
    return MG_OK;
}

void mg_process_destroy(mg_process *p) { free_proc(p); }

int mg_process_info(const mg_process *p, mg_info *o) {
    if (!p || !o) return MG_ERR_BAD_ARG;
    const mg_proc_table *t = p->tab;
    o->npar = t->npar;
    o->ngluon = t->ngluon;
    o->ndiagrams = t->ndiagrams;
    o->nterms = t->nterms;
    o->ncolor = t->ncolor;
    o->nhel = 1 << t->npar;
    o->ngood = p->ngood;
    o->nslot = t->nslot;
    o->nslot_top = t->nslot_top;
    o->nops = t->nops;
    o->njamp_updates = t->nscat;
    o->denom = t->denom;
    o->iden = t->iden;
    o->flops_diagram = t->flops_diagram;
    o->flops_colour = t->flops_colour;
    o->nchannel = t->nchannel;
    return MG_OK;
}

int mg_sde_channels(const mg_process *p, int *nchannel_out, int8_t *codes_out) {
    if (!p || (!nchannel_out && !codes_out)) return MG_ERR_BAD_ARG;
    const mg_proc_table *t = p->tab;
    if (nchannel_out) *nchannel_out = t->nchannel;
    if (codes_out) {
        memset(codes_out, 0, (size_t)t->nchannel * t->ncolor);
        for (int c = 0; c < t->nchannel; c++)
            for (int i = t->chan_off[c]; i < t->chan_off[c + 1]; i++)
                codes_out[(size_t)c * t->ncolor + (t->chan_flows[i] >> 3)] = (int8_t)(t->chan_flows[i] & 7);
    }
    return MG_OK;
}

int mg_color_matrix(const mg_process *p, int64_t *ints_out, int64_t *denom_out) {
    if (!p || !ints_out) return MG_ERR_BAD_ARG;
    const int nc = p->tab->ncolor;
    if (!p->tab->chat) {   // table-file process: C_st = row[rank of s^-1 t]
        const int ng = p->tab->ngluon;
        for (int a = 0; a < nc; a++) {
            int pos[16];
            for (int q = 0; q < ng; q++) pos[p->tab->cperm[a * ng + q]] = q;
            for (int b = 0; b < nc; b++) {
                long long rank = 0;
                unsigned used = 0;
                for (int q = 0; q < ng; q++) {
                    const int r = pos[p->tab->cperm[b * ng + q]];
                    int smaller = 0;
                    for (int x = 0; x < r; x++) smaller += !((used >> x) & 1u);
                    rank = rank * (ng - q) + smaller;
                    used |= 1u << r;
                }
                ints_out[(size_t)a * nc + b] = p->tab->crow[rank];
            }
        }
        if (denom_out) *denom_out = p->tab->denom;
        return MG_OK;
    }
    for (int i = 0; i < nc * nc; i++) ints_out[i] = p->tab->chat[i];
    if (denom_out) *denom_out = p->tab->denom;
    return MG_OK;
}

int mg_helicity_mask(const mg_process *p, uint8_t *mask_out) {
    if (!p || !mask_out) return MG_ERR_BAD_ARG;
    if (p->ngood < 0) return MG_ERR_NOT_FILTERED;
    memcpy(mask_out, p->mask, (size_t)1 << p->tab->npar);
    return MG_OK;
}

int mg_set_launch(mg_process *p, int tpe, int block) {
    if (!p) return MG_ERR_BAD_ARG;
    if (tpe) {
        if (tpe < 1 || tpe > 32 || (tpe & (tpe - 1))) return MG_ERR_BAD_ARG;
        p->tpe = tpe;
    }
    if (block) {   // the diagram kernel is compiled for blocks of at most 128 threads
        if (block < 32 || block > 128 || block % 32) return MG_ERR_BAD_ARG;
        p->block = block;
    }
    return MG_OK;
}

int mg_filter_helicities(mg_process *p, const double *mom, int64_t n, void *stream, int *ngood_out) {
    if (!p) return MG_ERR_BAD_ARG;
    if (n < 1 || n > 65536) return MG_ERR_BAD_ARG;
    int st = check_dev_ptr(mom, p->device);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int nhel = 1 << p->tab->npar;
    // evaluate every helicity: temporary list 0..nhel-1
    uint8_t all[512];
    memset(all, 1, sizeof(all));
    st = set_hel_list(p, all);
    if (st) return st;
    double *mh = nullptr;
    unsigned char *dmask = nullptr;
    uint8_t mask[512];
    cudaError_t e = cudaMalloc(&mh, sizeof(double) * n * nhel);
    if (e != cudaSuccess) {
        p->ngood = -1;
        return e == cudaErrorMemoryAllocation ? MG_ERR_NO_MEMORY : cuda_fail(e);
    }
    e = cudaMalloc(&dmask, nhel);
    if (e == cudaSuccess) e = cudaMemsetAsync(mh, 0, sizeof(double) * n * nhel, s);
    if (e == cudaSuccess) {
        if (p->big) {
            const int sb = sigmakin_big(p, mom, n, nullptr, mh, s);
            if (sb != MG_OK) {
                cudaFree(mh);
                cudaFree(dmask);
                p->ngood = -1;
                return sb;
            }
        } else {
            e = mg_launch_sigmakin(dev_view(p), mom, n, p->d_units, p->nunits, 32, p->block, nullptr,
                                   mh, s);
        }
    }
    if (e == cudaSuccess) e = mg_launch_helmask(mh, n, nhel, 1e-14, dmask, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mask, dmask, nhel, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(mh);
    cudaFree(dmask);
    if (e != cudaSuccess) {
        p->ngood = -1;
        return cuda_fail(e);
    }
    st = set_hel_list(p, mask);
    if (st) return st;
    if (ngood_out) *ngood_out = p->ngood;
    return MG_OK;
}

// Jamp buffer of a diagram launch over nevt events (tpe threads each): the
// jamps of every thread in global memory, updated by reductions at L2
// (mg_kernels.cu).  Grown on demand and kept; NULL (the jamps then stay in
// local memory) when it would exceed the limit (MG_JAMP_BUFFER_MAX, or the
// test hook's) or cannot be allocated; fp64_chunk keeps FP64 calls within it.
static const size_t MG_JAMP_BUFFER_MAX = 24ull << 30;

static size_t jamp_buffer_max(const mg_process *p) {
    return p->jg_max ? p->jg_max : MG_JAMP_BUFFER_MAX;
}

static double2 *jamp_buffer(mg_process *p, long long nevt, int tpe) {
    const long long threads = (nevt * tpe + p->block - 1) / p->block * p->block;
    const size_t bytes = (size_t)threads * 4 * p->tab->ncolor * sizeof(double2);
    if (p->jg_off || bytes > jamp_buffer_max(p)) return nullptr;
    if (bytes > p->jg_bytes) {
        cudaFree(p->d_jg);
        p->d_jg = nullptr;
        p->jg_bytes = 0;
        if (cudaMalloc(&p->d_jg, bytes) != cudaSuccess) {
            cudaGetLastError();   // out of memory is not sticky: run without
            p->d_jg = nullptr;
            return nullptr;
        }
        p->jg_bytes = bytes;
    }
    return p->d_jg;
}

// Events per FP64 diagram launch: all of them when their jamp buffer fits
// the buffer limit, else whole waves of the kernel's resident threads whose
// buffer does (the call then runs as several launches).
static long long fp64_chunk(mg_process *p, long long nevt, int tpe) {
    const long long per_event = (long long)tpe * 4 * p->tab->ncolor * (long long)sizeof(double2);
    const long long cap = (long long)jamp_buffer_max(p) / per_event - p->block;   // block rounding
    if (nevt <= cap || cap <= 0) return nevt;
    int nsm = 0, occ = 1;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess ||
        mg_sigmakin_occupancy(p->table_index, p->block, &occ) != MG_OK) {
        cudaGetLastError();
        return cap;
    }
    const long long wave = (long long)nsm * occ * p->block / tpe;   // events per wave
    return (wave > 0 && cap >= wave) ? cap / wave * wave : cap;
}

// Mixed precision: per chunk of events, the diagram kernel writes the jamps
// as BF16 GEMM rows, the tensor-core kernel forms the colour sums, and a small
// kernel adds each event's partial sums.  The chunk workspace is allocated on
// the first call and kept (the library owns it; freed by destroy).
static int sigmakin_mixed(mg_process *p, const double *mom, int64_t nevt, double *me, int tpe,
                          cudaStream_t s) {
    const int nup = pow2_at_least(p->nunits);
    const int cpe = 8 * nup;                                  // GEMM rows per event
    const long long row_bytes = 3LL * p->kp * 2;
    const long long ev_align = cpe < 128 ? 128 / cpe : 1;     // events per whole tile
    // chunk: whole waves of the diagram kernel (a partial last wave per chunk
    // idles SMs), at most 12 GiB of jamp rows
    int nsm = 0, occ = 1;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess ||
        mg_sigmakin_occupancy(p->table_index, p->block, &occ) != MG_OK)
        return MG_ERR_CUDA;
    long long wave = (long long)nsm * occ * p->block / tpe;
    wave = (wave + ev_align - 1) / ev_align * ev_align;
    const long long limit = (12LL << 30) / (row_bytes * cpe);
    long long chunk = limit / wave * wave;
    if (chunk < wave) chunk = limit / ev_align * ev_align;
    if (chunk < ev_align) chunk = ev_align;
    if (chunk > nevt) chunk = (nevt + ev_align - 1) / ev_align * ev_align;
    const long long rows = (chunk * cpe + 127) / 128 * 128;
    // more than 128 flows: the block-triangular kernel, one partial per row
    // and half of a 128-colour block
    const bool big_tc = p->tab->ncolor > 128;
    const int per_event = big_tc ? 0 : mg_tc_parts_per_event(cpe);
    const long long parts = big_tc ? rows * (2 * p->np / 128) : rows / 128 * mg_tc_parts_per_tile(cpe);
    if (rows > p->jbuf_rows) {
        cudaFree(p->d_jbuf);
        p->d_jbuf = nullptr;
        p->jbuf_rows = 0;
        cudaError_t e = cudaMalloc(&p->d_jbuf, rows * row_bytes);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? MG_ERR_NO_MEMORY : cuda_fail(e);
        p->jbuf_rows = rows;
        p->jbuf_nunits = -1;
    }
    if (p->jbuf_nunits != p->nunits) {  // rows of padding units must read as zero
        MG_CUDA(cudaMemsetAsync(p->d_jbuf, 0, p->jbuf_rows * row_bytes, s));
        p->jbuf_nunits = p->nunits;
    }
    if (parts > p->part_len) {
        cudaFree(p->d_part);
        p->d_part = nullptr;
        p->part_len = 0;
        cudaError_t e = cudaMalloc(&p->d_part, parts * sizeof(double));
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? MG_ERR_NO_MEMORY : cuda_fail(e);
        p->part_len = parts;
    }
    double2 *jg = jamp_buffer(p, chunk < nevt ? chunk : nevt, tpe);
    const mg_dev_proc dp = dev_view(p);
    for (long long e0 = 0; e0 < nevt; e0 += chunk) {
        const long long n = (nevt - e0 < chunk) ? nevt - e0 : chunk;
        const long long used = (n * cpe + 127) / 128 * 128;
        int slot = mg_timer_begin(p, s, MG_KT_DIAGRAM);
        MG_CUDA(mg_launch_sigmakin(dp, mom + e0 * p->tab->npar * 4, n, p->d_units, p->nunits, tpe,
                                   p->block, nullptr, nullptr, s, p->d_jbuf, p->kp, nup, nullptr, jg));
        mg_timer_end(p, s, slot);
        slot = mg_timer_begin(p, s, MG_KT_COLOUR);
        if (big_tc)
            MG_CUDA(mg_launch_colorsum_tc_big(p->d_jbuf, used, p->kp, p->d_cmat, p->np,
                                              p->debug_extra_tx, p->d_part, p->d_err, s));
        else
            MG_CUDA(mg_launch_colorsum_tc(p->d_jbuf, used, p->kp, p->d_cmat, p->np, p->tab->ncolor,
                                          cpe, p->debug_extra_tx, p->d_part, p->d_err, s));
        mg_timer_end(p, s, slot);
        slot = mg_timer_begin(p, s, MG_KT_EVENT_SUM);
        if (big_tc)
            MG_CUDA(mg_launch_event_sum_rows(p->d_part, used, 2 * p->np / 128, cpe, n, p->factor,
                                             me + e0, s));
        else
            MG_CUDA(mg_launch_event_sum(p->d_part, n, per_event, p->factor, me + e0, s));
        mg_timer_end(p, s, slot);
    }
    return MG_OK;
}

static int sigmakin_impl(mg_process *p, const double *mom, int64_t nevt, double *me,
                         double *me_hel, void *stream) {
    if (!p) return MG_ERR_BAD_ARG;
    if (nevt < 0) return MG_ERR_BAD_ARG;
    if (p->ngood < 0) return MG_ERR_NOT_FILTERED;
    if (nevt == 0) return MG_OK;
    int st = check_dev_ptr(mom, p->device);
    if (st) return st;
    if (me && (st = check_dev_ptr(me, p->device))) return st;
    if (me_hel && (st = check_dev_ptr(me_hel, p->device))) return st;
    if (!me && !me_hel) return MG_ERR_BAD_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int nhel = 1 << p->tab->npar;
    if (me_hel) MG_CUDA(cudaMemsetAsync(me_hel, 0, sizeof(double) * nevt * nhel, s));
    if (p->ngood == 0) {
        if (me) MG_CUDA(cudaMemsetAsync(me, 0, sizeof(double) * nevt, s));
        return MG_OK;
    }
    int tpe = p->tpe;
    while (tpe > 1 && tpe > p->nunits) tpe >>= 1;
    if (p->big) return sigmakin_big(p, mom, nevt, me, me_hel, s);
    if (p->par.precision == MG_MIXED_BF16) {
        if (me_hel) return MG_ERR_UNSUPPORTED;
        return sigmakin_mixed(p, mom, nevt, me, tpe, s);
    }
    const long long chunk = fp64_chunk(p, nevt, tpe);
    double2 *jg = jamp_buffer(p, chunk, tpe);
    const int npar = p->tab->npar;
    for (long long e0 = 0; e0 < nevt; e0 += chunk) {
        const long long n = nevt - e0 < chunk ? nevt - e0 : chunk;
        const int slot = mg_timer_begin(p, s, MG_KT_DIAGRAM);
        MG_CUDA(mg_launch_sigmakin(dev_view(p), mom + e0 * npar * 4, n, p->d_units, p->nunits, tpe,
                                   p->block, me ? me + e0 : nullptr, me_hel ? me_hel + e0 * nhel : nullptr,
                                   s, nullptr, 0, 0, nullptr, jg));
        mg_timer_end(p, s, slot);
    }
    return MG_OK;
}

int mg_sigmakin(mg_process *p, const double *mom, int64_t nevt, double *me, void *stream) {
    if (p && nevt == 0 && p->ngood >= 0) return MG_OK;
    if (!me) return MG_ERR_BAD_ARG;
    return sigmakin_impl(p, mom, nevt, me, nullptr, stream);
}

int mg_sigmakin_hel(mg_process *p, const double *mom, int64_t nevt, double *me, double *me_hel,
                    void *stream) {
    if (p && nevt == 0 && p->ngood >= 0) return MG_OK;
    if (!me_hel) return MG_ERR_BAD_ARG;
    return sigmakin_impl(p, mom, nevt, me, me_hel, stream);
}

int mg_set_kernel_timing(mg_process *p, int max_launches) {
    if (!p || max_launches < 0) return MG_ERR_BAD_ARG;
    for (int i = 0; i < 2 * p->tcap; i++) cudaEventDestroy(p->tev[i]);
    free(p->tev);
    free(p->tkind);
    p->tev = nullptr;
    p->tkind = nullptr;
    p->tcap = p->tn = p->tdropped = 0;
    p->timing = 0;
    if (max_launches == 0) return MG_OK;
    p->tev = static_cast<cudaEvent_t *>(calloc(2 * (size_t)max_launches, sizeof(cudaEvent_t)));
    p->tkind = static_cast<int *>(calloc((size_t)max_launches, sizeof(int)));
    if (!p->tev || !p->tkind) return MG_ERR_NO_MEMORY;
    for (int i = 0; i < 2 * max_launches; i++) {
        cudaError_t e = cudaEventCreate(&p->tev[i]);
        if (e != cudaSuccess) {
            p->tcap = i / 2;   // pairs fully created so far are destroyed later
            for (int j = 2 * p->tcap; j < i; j++) cudaEventDestroy(p->tev[j]);
            return cuda_fail(e);
        }
    }
    p->tcap = max_launches;
    p->timing = 1;
    return MG_OK;
}

int mg_kernel_times(mg_process *p, int reset, double *ms_out, int *launches_out) {
    if (!p || !ms_out || !launches_out) return MG_ERR_BAD_ARG;
    for (int k = 0; k < MG_KT_NKIND; k++) {
        ms_out[k] = 0.0;
        launches_out[k] = 0;
    }
    if (p->tdropped) return MG_ERR_UNSUPPORTED;
    if (p->tn > 0) MG_CUDA(cudaEventSynchronize(p->tev[2 * p->tn - 1]));
    for (int i = 0; i < p->tn; i++) {
        float ms = 0.0f;
        MG_CUDA(cudaEventElapsedTime(&ms, p->tev[2 * i], p->tev[2 * i + 1]));
        ms_out[p->tkind[i]] += ms;
        launches_out[p->tkind[i]] += 1;
    }
    if (reset) p->tn = 0;
    return MG_OK;
}

}  // extern "C"

static std::atomic<unsigned long long> g_launches{0};

void mg_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" int mg_launch_count(unsigned long long *out) {
    if (!out) return MG_ERR_BAD_ARG;
    *out = g_launches.load(std::memory_order_relaxed);
    return MG_OK;
}

int mg_timer_begin(mg_process *p, cudaStream_t s, int kind) {
    if (!p->timing) return -1;
    if (p->tn >= p->tcap) {
        p->tdropped = 1;
        return -1;
    }
    const int slot = p->tn++;
    p->tkind[slot] = kind;
    if (cudaEventRecord(p->tev[2 * slot], s) != cudaSuccess) p->tdropped = 1;
    return slot;
}

void mg_timer_end(mg_process *p, cudaStream_t s, int slot) {
    if (slot < 0) return;
    if (cudaEventRecord(p->tev[2 * slot + 1], s) != cudaSuccess) p->tdropped = 1;
}

// ---------------------------------------------------------------------------
// Helicity filter without device allocations.
//
// mg_filter_helicities allocates (cudaMalloc) and frees (cudaFree, which
// synchronises the whole device) a scratch buffer on every call.  The variant
// below takes that scratch from a fixed array compiled into the library
// instead: room for MG_NOALLOC_FILTER_MAX_EVENTS test events x 256 helicities
// of |M_h|^2 (FP64) plus a 256-byte mask, 128.25 KiB in total, held on every
// GPU that loads the library until the process exits.
#define MG_NOALLOC_FILTER_MAX_EVENTS 64
#define MG_NOALLOC_MAX_DEVICES 64
static __device__ __align__(256) unsigned char
    g_filter_scratch[MG_NOALLOC_FILTER_MAX_EVENTS * 256 * sizeof(double) + 256];

namespace {
std::mutex g_scratch_mu;
void *g_scratch_addr[MG_NOALLOC_MAX_DEVICES];  // device address of g_filter_scratch, per device

// Device address of the scratch array on the current device.  The host-side
// name g_filter_scratch is only a stand-in; kernels must get this address.
int scratch_address(int device, void **out) {
    if (device < 0 || device >= MG_NOALLOC_MAX_DEVICES) return MG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_filter_scratch);
        if (e != cudaSuccess) return cuda_fail(e);
        g_scratch_addr[device] = ptr;
    }
    *out = g_scratch_addr[device];
    return MG_OK;
}
}  // namespace

extern "C" int mg_filter_helicities_noalloc(mg_process *p, const double *mom, int64_t n,
                                            void *stream, int *ngood_out) {
    if (!p) return MG_ERR_BAD_ARG;
    if (n < 1 || n > MG_NOALLOC_FILTER_MAX_EVENTS) return MG_ERR_BAD_ARG;
    if (p->big) return MG_ERR_UNSUPPORTED;   // 512 helicities exceed the fixed scratch
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return MG_ERR_CUDA;
    if (cur != p->device) return MG_ERR_BAD_ARG;
    int st = check_dev_ptr(mom, p->device);
    if (st) return st;
    void *scratch = nullptr;
    st = scratch_address(cur, &scratch);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int nhel = 1 << p->tab->npar;
    double *mh = (double *)scratch;
    unsigned char *dmask = (unsigned char *)scratch + MG_NOALLOC_FILTER_MAX_EVENTS * 256 * sizeof(double);
    uint8_t all[512];
    memset(all, 1, sizeof(all));
    // unit-list uploads ordered on the caller's stream (no legacy-stream copy)
    st = set_hel_list(p, all, true, s);
    if (st) return st;
    uint8_t mask[512];
    // the array keeps the previous call's contents: clear what is read
    cudaError_t e = cudaMemsetAsync(mh, 0, sizeof(double) * n * nhel, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dmask, 0, nhel, s);
    if (e == cudaSuccess)
        e = mg_launch_sigmakin(dev_view(p), mom, n, p->d_units, p->nunits, 32, p->block, nullptr, mh, s);
    if (e == cudaSuccess) e = mg_launch_helmask(mh, n, nhel, 1e-14, dmask, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mask, dmask, nhel, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        p->ngood = -1;
        return cuda_fail(e);
    }
    st = set_hel_list(p, mask, true, s);
    if (st) return st;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (ngood_out) *ngood_out = p->ngood;
    return MG_OK;
}

// ---------------------------------------------------------------------------
int mg_check_dev_ptr(const void *ptr, int device) { return check_dev_ptr(ptr, device); }
int mg_cuda_fail(cudaError_t e) { return cuda_fail(e); }
mg_dev_proc mg_dev_view(const mg_process *p) { return dev_view(p); }

// Test hook: the tensor-core colour sum of caller rows, per group of 8 rows.
extern "C" int mg_debug_colour_sum_rows(mg_process *p, const double *rows, int64_t nrows,
                                        double *q8, void *stream) {
    if (!p || nrows <= 0 || nrows % 128) return MG_ERR_BAD_ARG;
    if (p->par.precision != MG_MIXED_BF16 || !p->d_cmat) return MG_ERR_UNSUPPORTED;
    int st = check_dev_ptr(rows, p->device);
    if (!st) st = check_dev_ptr(q8, p->device);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int nc = p->tab->ncolor;
    const bool block = nc > 128;
    __nv_bfloat16 *jb = nullptr;
    double *part = nullptr;
    const long long nparts = block ? nrows * (2 * p->np / 128) : nrows / 128 * mg_tc_parts_per_tile(8);
    cudaError_t e = cudaMalloc(&jb, sizeof(__nv_bfloat16) * 3 * p->kp * nrows);
    if (e == cudaSuccess) e = cudaMalloc(&part, sizeof(double) * nparts);
    if (e == cudaSuccess) e = mg_launch_rows_split(rows, nrows, nc, p->kp, jb, s);
    if (e == cudaSuccess) {
        if (block)
            e = mg_launch_colorsum_tc_big(jb, nrows, p->kp, p->d_cmat, p->np, 0, part, p->d_err, s);
        else
            e = mg_launch_colorsum_tc(jb, nrows, p->kp, p->d_cmat, p->np, nc, 8, 0, part, p->d_err, s);
    }
    if (e == cudaSuccess) {
        if (block)
            e = mg_launch_event_sum_rows(part, nrows, 2 * p->np / 128, 8, nrows / 8, 1.0, q8, s);
        else
            e = mg_launch_event_sum(part, nrows / 8, mg_tc_parts_per_event(8), 1.0, q8, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(jb);
    cudaFree(part);
    return e == cudaSuccess ? MG_OK : cuda_fail(e);
}

extern "C" int mg_device_status(mg_process *p, void *stream) {
    if (!p) return MG_ERR_BAD_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    MG_CUDA(cudaStreamSynchronize(s));
    MG_CUDA(cudaMemcpy(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        MG_CUDA(cudaMemset(p->d_err, 0, sizeof(int)));
        return MG_ERR_DEVICE_TIMEOUT;
    }
    return MG_OK;
}

extern "C" int mg_debug_inject_stall(mg_process *p, unsigned int extra_bytes) {
    if (!p) return MG_ERR_BAD_ARG;
    p->debug_extra_tx = extra_bytes;
    return MG_OK;
}

extern "C" int mg_debug_jamp_buffer(mg_process *p, int enable, int64_t max_bytes) {
    if (!p || max_bytes < 0) return MG_ERR_BAD_ARG;
    p->jg_off = enable ? 0 : 1;
    p->jg_max = (size_t)max_bytes;
    return MG_OK;
}

// Per-event extras of the FP64 path (see mgpu.h): running alpha_s, single-
// diagram-enhancement weight, helicity-summed flow weights, helicity and
// colour choice.
extern "C" int mg_sigmakin_ex(mg_process *p, const double *mom, int64_t nevt,
                              const mg_sigmakin_extras *x, double *me, void *stream) {
    if (!p || !x || nevt < 0) return MG_ERR_BAD_ARG;
    if (p->ngood < 0) return MG_ERR_NOT_FILTERED;
    if (p->par.precision != MG_FP64 && !p->big) return MG_ERR_UNSUPPORTED;
    if (nevt == 0) return MG_OK;
    int st = check_dev_ptr(mom, p->device);
    if (!st && me) st = check_dev_ptr(me, p->device);
    if (!st && x->alphas_dev) st = check_dev_ptr(x->alphas_dev, p->device);
    if (!st && x->sde_weight_dev) st = check_dev_ptr(x->sde_weight_dev, p->device);
    if (!st && x->flow_weight_dev) st = check_dev_ptr(x->flow_weight_dev, p->device);
    if (!st && x->channel_ids_dev) st = check_dev_ptr(x->channel_ids_dev, p->device, 4);
    if (st) return st;
    const bool want_hel = x->hel_out_dev && x->rnd_hel_dev;
    const bool want_col = x->col_out_dev && x->rnd_col_dev;
    if ((x->hel_out_dev && !x->rnd_hel_dev) || (x->col_out_dev && !x->rnd_col_dev)) return MG_ERR_BAD_ARG;
    const bool want_sde = x->channel >= 0 || x->channel_ids_dev;
    if (want_sde && !x->sde_weight_dev) return MG_ERR_BAD_ARG;
    if (x->channel < -1 || x->channel >= p->tab->nchannel) return MG_ERR_BAD_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int nhel = 1 << p->tab->npar, nc = p->tab->ncolor;
    if ((want_hel || (want_col && !x->flow_weight_dev)) && nevt > p->sel_cap) {
        cudaFree(p->d_sel_hel);
        cudaFree(p->d_sel_jw);
        p->d_sel_hel = nullptr;
        p->d_sel_jw = nullptr;
        p->sel_cap = 0;
        cudaError_t e = cudaMalloc(&p->d_sel_hel, sizeof(double) * nevt * nhel);
        if (e == cudaSuccess) e = cudaMalloc(&p->d_sel_jw, sizeof(double) * nevt * nc);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? MG_ERR_NO_MEMORY : cuda_fail(e);
        p->sel_cap = nevt;
    }
    double *mh = want_hel ? p->d_sel_hel : nullptr;
    double *jw = x->flow_weight_dev ? x->flow_weight_dev : (want_col ? p->d_sel_jw : nullptr);
    if (mh) MG_CUDA(cudaMemsetAsync(mh, 0, sizeof(double) * nevt * nhel, s));
    if (p->big) {   // table-file process: extras from the chunked HBM pipeline
        const BigExtras bx = {x->alphas_dev, x->channel, x->channel_ids_dev,
                              want_sde ? x->sde_weight_dev : nullptr, jw};
        if (!me && !mh && !jw && !want_sde) return MG_OK;
        st = sigmakin_big(p, mom, nevt, me, mh, s, &bx);
        if (st) return st;
        if (want_hel || want_col)
            MG_CUDA(mg_launch_select(mh, nhel, jw, nc, nevt, x->rnd_hel_dev, x->rnd_col_dev,
                                     want_hel ? x->hel_out_dev : nullptr, want_col ? x->col_out_dev : nullptr,
                                     s));
        return MG_OK;
    }
    mg_extras ex;
    ex.alphas = x->alphas_dev;
    ex.alphas0 = p->par.alphas;
    ex.channel = x->channel;
    ex.channel_ids = x->channel_ids_dev;
    ex.sde = want_sde ? x->sde_weight_dev : nullptr;
    ex.jw = jw;
    int tpe = p->tpe;
    while (tpe > 1 && tpe > p->nunits) tpe >>= 1;
    const long long chunk = fp64_chunk(p, nevt, tpe);
    double2 *jg = jamp_buffer(p, chunk, tpe);
    for (long long e0 = 0; e0 < nevt; e0 += chunk) {
        const long long n = nevt - e0 < chunk ? nevt - e0 : chunk;
        mg_extras exc = ex;   // the chunk's slice of every per-event array
        if (exc.alphas) exc.alphas += e0;
        if (exc.channel_ids) exc.channel_ids += e0;
        if (exc.sde) exc.sde += e0;
        if (exc.jw) exc.jw += e0 * nc;
        MG_CUDA(mg_launch_sigmakin(dev_view(p), mom + e0 * p->tab->npar * 4, n, p->d_units, p->nunits,
                                   tpe, p->block, me ? me + e0 : nullptr, mh ? mh + e0 * nhel : nullptr, s,
                                   nullptr, 0, 0, &exc, jg));
    }
    if (want_hel || want_col)
        MG_CUDA(mg_launch_select(mh, nhel, jw, nc, nevt, x->rnd_hel_dev, x->rnd_col_dev,
                                 want_hel ? x->hel_out_dev : nullptr, want_col ? x->col_out_dev : nullptr, s));
    return MG_OK;
}
