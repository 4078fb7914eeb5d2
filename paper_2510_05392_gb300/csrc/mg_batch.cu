// Uneven multi-process batch: plan, CUDA-graph replay and autotuner (host).
//
// The paper runs one process per application, notes that several processes
// can share a GPU (Sec. 2.3), shows that a GPU needs enough independent work
// per launch to reach its peak (Sec. 3.1) and captures repeated kernel
// sequences in CUDA graphs (Sec. 4.1, "gpuDiagrams").  A batch here is a list
// of event blocks of different processes evaluated by ONE persistent launch
// (k_batch in mg_kernels.cu): warps take 32-slot chunks from an atomic
// counter, heaviest process first.  The launch (counter reset + kernel) is
// captured once in a CUDA graph and replayed by mg_batch_run; the autotuner
// picks the threads per event of every block and the CTAs per SM of the
// persistent grid by timing the batch itself.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "mg_process.h"
#include "mgpu.h"

struct mg_batch {
    int n;
    std::vector<mg_batch_item> items;   // host copy, sorted heaviest first
    std::vector<int> order;             // items[k] came from caller index order[k]
    mg_batch_item *d_items;
    int *d_units;                       // the blocks' work-unit lists, copied at creation
    unsigned long long *d_counter;
    double2 *d_jg;                      // jamp buffers of the persistent kernel's threads
    int max_ncolor;                     // largest colour-flow count of the items
    long long total_slots;
    int nsm, ctas_per_sm, max_ctas_per_sm;
    int device;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace {

void layout(mg_batch *b) {
    long long s = 0;
    for (auto &it : b->items) {
        it.slot_begin = s;
        const long long slots = it.nevt * it.tpe;
        s += (slots + 31) / 32 * 32;
        it.slot_end = s;
    }
    b->total_slots = s;
}

int upload(mg_batch *b) {
    layout(b);
    cudaError_t e = cudaMemcpy(b->d_items, b->items.data(), sizeof(mg_batch_item) * b->n,
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return mg_cuda_fail(e);
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    return MG_OK;
}

int launch(mg_batch *b, cudaStream_t s) {
    cudaError_t e = mg_launch_batch(b->d_items, b->n, b->d_counter, b->total_slots,
                                    b->nsm * b->ctas_per_sm, s, b->d_jg);
    return e == cudaSuccess ? MG_OK : mg_cuda_fail(e);
}

void free_batch(mg_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_items);
    cudaFree(b->d_units);
    cudaFree(b->d_counter);
    cudaFree(b->d_jg);
    delete b;
}

}  // namespace

extern "C" {

int mg_batch_create(int nproc, mg_process *const *procs, const double *const *mom,
                    const int64_t *nevt, double *const *me_out, mg_batch **out) {
    if (!out || nproc < 1 || nproc > 64 || !procs || !mom || !nevt || !me_out) return MG_ERR_BAD_ARG;
    *out = nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return MG_ERR_CUDA;
    mg_batch *b = new mg_batch();
    b->n = nproc;
    b->device = dev;
    for (int i = 0; i < nproc; i++) {
        mg_process *p = procs[i];
        if (!p || nevt[i] < 0 || p->device != dev) {
            free_batch(b);
            return MG_ERR_BAD_ARG;
        }
        if (p->ngood < 0) {
            free_batch(b);
            return MG_ERR_NOT_FILTERED;
        }
        if (p->tab->ngluon > MG_BATCH_MAX_NGLUON || p->par.precision != MG_FP64) {
            free_batch(b);
            return MG_ERR_UNSUPPORTED;
        }
        if (nevt[i] > 0) {
            int st = mg_check_dev_ptr(mom[i], dev);
            if (!st) st = mg_check_dev_ptr(me_out[i], dev);
            if (st) {
                free_batch(b);
                return st;
            }
        }
        const mg_dev_proc dp = mg_dev_view(p);
        mg_batch_item it;
        memset(&it, 0, sizeof(it));
        it.ops = dp.ops;
        it.scat = dp.scat;
        it.cup = dp.cup;
        it.units = p->d_units;
        it.mom = mom[i];
        it.me = me_out[i];
        it.nevt = nevt[i];
        it.mt = dp.mt;
        it.wt = dp.wt;
        it.factor = dp.factor;
        it.nops = dp.nops;
        it.nunits = p->nunits;
        int tpe = p->tpe;
        while (tpe > 1 && tpe > p->nunits) tpe >>= 1;
        it.tpe = tpe;
        it.table_index = dp.table_index;
        if (p->tab->ncolor > b->max_ncolor) b->max_ncolor = p->tab->ncolor;
        b->items.push_back(it);
        b->order.push_back(i);
    }
    // heaviest process first (longest-processing-time order)
    std::vector<int> idx(nproc);
    for (int i = 0; i < nproc; i++) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) {
        return b->items[a].table_index > b->items[c].table_index;
    });
    std::vector<mg_batch_item> sorted;
    std::vector<int> ord;
    for (int k : idx) {
        sorted.push_back(b->items[k]);
        ord.push_back(b->order[k]);
    }
    b->items = sorted;
    b->order = ord;
    if (cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        mg_batch_ctas_per_sm(&b->max_ctas_per_sm) != MG_OK) {
        free_batch(b);
        return MG_ERR_CUDA;
    }
    if (b->max_ctas_per_sm < 1) b->max_ctas_per_sm = 1;
    b->ctas_per_sm = b->max_ctas_per_sm;
    cudaError_t e = cudaMalloc(&b->d_items, sizeof(mg_batch_item) * nproc);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(unsigned long long));
    // jamp buffers for the largest grid the autotuner may launch (jamp
    // updates as L2 reductions, as in mg_sigmakin)
    if (e == cudaSuccess && b->max_ncolor > 0)
        e = cudaMalloc(&b->d_jg, sizeof(double2) * 4 * (size_t)b->max_ncolor *
                                     (size_t)b->nsm * b->max_ctas_per_sm * 128);
    // the batch's own copy of every block's work-unit list (at most 128 units
    // each), so that a later helicity filter of a process does not change the
    // captured launch under it
    if (e == cudaSuccess) e = cudaMalloc(&b->d_units, sizeof(int) * 128 * nproc);
    for (int k = 0; e == cudaSuccess && k < nproc; k++) {
        e = cudaMemcpy(b->d_units + 128 * k, b->items[k].units, sizeof(int) * b->items[k].nunits,
                       cudaMemcpyDeviceToDevice);
        b->items[k].units = b->d_units + 128 * k;
    }
    if (e != cudaSuccess) {
        free_batch(b);
        return e == cudaErrorMemoryAllocation ? MG_ERR_NO_MEMORY : mg_cuda_fail(e);
    }
    int st = upload(b);
    if (st) {
        free_batch(b);
        return st;
    }
    *out = b;
    return MG_OK;
}

int mg_batch_run(mg_batch *b, void *stream) {
    if (!b) return MG_ERR_BAD_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!b->exec) {
        // capture the launch once (a private stream: the legacy default stream
        // cannot be captured), replay it afterwards
        cudaStream_t cs;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return mg_cuda_fail(e);
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const int st = launch(b, cs);
            cudaGraph_t g = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
            if (st != MG_OK) {
                if (g) cudaGraphDestroy(g);
                cudaStreamDestroy(cs);
                return st;
            }
            e = e2;
            if (e == cudaSuccess) {
                b->graph = g;
                e = cudaGraphInstantiate(&b->exec, g, 0);
            }
        }
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return mg_cuda_fail(e);
    }
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    return e == cudaSuccess ? MG_OK : mg_cuda_fail(e);
}

int mg_batch_autotune(mg_batch *b, void *stream, int reps, double *best_ms_out) {
    if (!b || reps < 1) return MG_ERR_BAD_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return MG_ERR_CUDA;
    int st = MG_OK;
    auto timeit = [&](double *ms) -> int {
        int r = upload(b);
        if (r) return r;
        if ((r = launch(b, s))) return r;  // warm-up
        cudaEventRecord(e0, s);
        for (int i = 0; i < reps; i++)
            if ((r = launch(b, s))) return r;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return MG_ERR_CUDA;
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        *ms = f / reps;
        return MG_OK;
    };
    double best = 0.0;
    st = timeit(&best);
    // coordinate descent: threads per event of each block, then CTAs per SM
    for (int k = 0; k < b->n && st == MG_OK; k++) {
        const int keep = b->items[k].tpe;
        int best_t = keep;
        for (int t = 1; t <= 16 && st == MG_OK; t <<= 1) {
            if (t == keep || t > b->items[k].nunits || b->items[k].nevt == 0) continue;
            b->items[k].tpe = t;
            double ms = 0.0;
            st = timeit(&ms);
            if (st == MG_OK && ms < best) {
                best = ms;
                best_t = t;
            }
        }
        b->items[k].tpe = best_t;
    }
    const int keep_c = b->ctas_per_sm;
    int best_c = keep_c;
    for (int c = 1; c <= b->max_ctas_per_sm && st == MG_OK; c++) {
        if (c == keep_c) continue;
        b->ctas_per_sm = c;
        double ms = 0.0;
        st = timeit(&ms);
        if (st == MG_OK && ms < best) {
            best = ms;
            best_c = c;
        }
    }
    b->ctas_per_sm = best_c;
    if (st == MG_OK) st = upload(b);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == MG_OK && best_ms_out) *best_ms_out = best;
    return st;
}

int mg_batch_config(const mg_batch *b, int *tpe_out, int *ctas_per_sm_out) {
    if (!b) return MG_ERR_BAD_ARG;
    if (tpe_out)
        for (int k = 0; k < b->n; k++) tpe_out[b->order[k]] = b->items[k].tpe;
    if (ctas_per_sm_out) *ctas_per_sm_out = b->ctas_per_sm;
    return MG_OK;
}

void mg_batch_destroy(mg_batch *b) { free_batch(b); }

int mg_sigmakin_batch(int nproc, mg_process *const *procs, const double *const *mom,
                      const int64_t *nevt, double *const *me_out, void *stream) {
    mg_batch *b = nullptr;
    int st = mg_batch_create(nproc, procs, mom, nevt, me_out, &b);
    if (st) return st;
    st = launch(b, (cudaStream_t)stream);
    // the plan's device arrays must outlive the launch
    if (st == MG_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) st = MG_ERR_CUDA;
    free_batch(b);
    return st;
}

}  // extern "C"
