// batch.cu -- step A8: many independent problems of uneven size in one
// graph launch.  Each problem has its own plan (problems with identical
// geometry share kernel spectra); plans are spread round-robin over worker
// streams; the whole batch is captured once into a CUDA graph that forks from
// the launch stream to the workers and joins back, and is replayed with one
// cudaGraphLaunch while the arguments stay the same.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <new>
#include <vector>

#include "sdf_internal.cuh"

using namespace sdf;

struct sdf_batch_s {
    int n = 0, D = 0;
    std::vector<sdf_plan> plans;
    std::vector<cudaStream_t> workers;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr, done = nullptr;
    cudaStream_t stream = nullptr;   // the caller's stream (may be the legacy stream)
    cudaStream_t origin = nullptr;   // internal stream the graph is captured on
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // arguments the graph was captured with
    std::vector<int64_t> K;
    std::vector<const void *> ptrs;
};

static void batch_free(sdf_batch_s *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto s : b->workers) cudaStreamSynchronize(s);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    // plans that share spectra first, owners last
    for (int pass = 0; pass < 2; ++pass)
        for (auto &p : b->plans)
            if (p && (p->shares_spectra == (pass == 0))) {
                sdf_plan_destroy(p);
                p = nullptr;
            }
    for (auto s : b->workers) cudaStreamDestroy(s);
    for (auto e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    if (b->origin) cudaStreamDestroy(b->origin);
}

static sdf_status fail(cudaError_t e) {
    set_last_error(cudaGetErrorString(e));
    cudaGetLastError();  // do not leave the error for the next call to find
    return e == cudaErrorMemoryAllocation ? SDF_ERR_OOM : SDF_ERR_CUDA;
}

extern "C" {

sdf_status sdf_batch_create(sdf_batch *out, int n, int D, const int64_t *dims, const double *h, const double *tau,
                            int precision, unsigned outputs, int n_streams, void *stream) {
    if (!out) return SDF_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || !dims || !h || !tau || n_streams < 1 || n_streams > 32) return SDF_ERR_INVALID_ARG;
    if (D != 2 && D != 3) return SDF_ERR_UNSUPPORTED;  // 1D plans are one CTA each: no batch
    sdf_batch_s *b = new (std::nothrow) sdf_batch_s();
    if (!b) return SDF_ERR_OOM;
    b->n = n;
    b->D = D;
    b->stream = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    for (int s = 0; s < n_streams; ++s) {
        cudaStream_t st;
        cudaEvent_t ev;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
            batch_free(b);
            delete b;
            return fail(e);
        }
        b->workers.push_back(st);
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
            batch_free(b);
            delete b;
            return fail(e);
        }
        b->join.push_back(ev);
    }
    if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking)) != cudaSuccess) {
        batch_free(b);
        delete b;
        return fail(e);
    }
    b->plans.assign(n, nullptr);
    for (int i = 0; i < n; ++i) {
        // an earlier problem with the same geometry owns the spectra
        const sdf_plan_impl *share = nullptr;
        for (int j = 0; j < i && !share; ++j) {
            bool same = h[j] == h[i] && tau[j] == tau[i];
            for (int a = 0; a < D; ++a) same = same && dims[j * D + a] == dims[i * D + a];
            if (same && !b->plans[j]->shares_spectra) share = b->plans[j];
        }
        sdf_status s = plan_create_shared(&b->plans[i], D, dims + (int64_t)i * D, h[i], tau[i], precision, outputs,
                                          b->workers[i % n_streams], share);
        if (s != SDF_OK) {
            batch_free(b);
            delete b;
            return s;
        }
    }
    *out = b;
    return SDF_OK;
}

static const void *at(const void *const *arr, int i) { return arr ? arr[i] : nullptr; }

sdf_status sdf_batch_execute(sdf_batch b, const int64_t *K, const double *const *points, const double *const *weights,
                             void *const *S, void *const *dS, void *const *d2S, int8_t *const *sign,
                             uint8_t *const *flags) {
    if (!b || !K || !points) return SDF_ERR_INVALID_ARG;
    const int n = b->n;
    std::vector<const void *> ptrs;
    ptrs.reserve(7 * n);
    for (int i = 0; i < n; ++i) {
        ptrs.push_back(points[i]);
        ptrs.push_back(at((const void *const *)weights, i));
        ptrs.push_back(at((const void *const *)S, i));
        ptrs.push_back(at((const void *const *)dS, i));
        ptrs.push_back(at((const void *const *)d2S, i));
        ptrs.push_back(at((const void *const *)sign, i));
        ptrs.push_back(at((const void *const *)flags, i));
    }
    std::vector<int64_t> kv(K, K + n);
    auto run_all = [&]() -> sdf_status {
        for (int i = 0; i < n; ++i) {
            sdf_status s = sdf_execute(b->plans[i], K[i], points[i], weights ? weights[i] : nullptr,
                                       S ? S[i] : nullptr, dS ? dS[i] : nullptr, d2S ? d2S[i] : nullptr,
                                       sign ? sign[i] : nullptr, flags ? flags[i] : nullptr);
            if (s != SDF_OK) return s;
        }
        return SDF_OK;
    };
    cudaError_t e;
    if (!b->exec || kv != b->K || ptrs != b->ptrs) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        if (b->graph) {
            cudaGraphDestroy(b->graph);
            b->graph = nullptr;
        }
        // one plain run: sizes point buffers and sets kernel attributes, so
        // the captured run performs no allocation or synchronisation
        if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return fail(e);
        sdf_status s = run_all();
        if (s != SDF_OK) return s;
        for (auto st : b->workers)
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
        if ((e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return fail(e);
        if ((e = cudaEventRecord(b->fork, b->origin)) == cudaSuccess) {
            for (auto st : b->workers)
                if ((e = cudaStreamWaitEvent(st, b->fork, 0)) != cudaSuccess) break;
        }
        if (e == cudaSuccess) s = run_all();
        if (e == cudaSuccess && s == SDF_OK) {
            for (size_t w = 0; w < b->workers.size(); ++w) {
                if ((e = cudaEventRecord(b->join[w], b->workers[w])) != cudaSuccess) break;
                if ((e = cudaStreamWaitEvent(b->origin, b->join[w], 0)) != cudaSuccess) break;
            }
        }
        cudaGraph_t g = nullptr;
        cudaError_t ee = cudaStreamEndCapture(b->origin, &g);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(e);
        }
        if (s != SDF_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (ee != cudaSuccess) return fail(ee);
        b->graph = g;
        if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) return fail(e);
        b->K = kv;
        b->ptrs = ptrs;
    }
    if ((e = cudaGraphLaunch(b->exec, b->stream)) != cudaSuccess) return fail(e);
    return SDF_OK;
}

sdf_status sdf_batch_autotune(sdf_batch b, const int64_t *K, const double *const *points,
                              const double *const *weights, int reps) {
    if (!b || !K || !points || reps < 1) return SDF_ERR_INVALID_ARG;
    const int n = b->n;
    cudaError_t e;
    if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return fail(e);
    // the owner of each problem's spectra: the first problem of its geometry
    std::vector<int> owner(n, -1);
    for (int i = 0; i < n; ++i) {
        if (!b->plans[i]->shares_spectra) {
            owner[i] = i;
            continue;
        }
        for (int j = 0; j < i && owner[i] < 0; ++j) {
            sdf_plan pj = b->plans[j], pi = b->plans[i];
            bool same = !pj->shares_spectra && pj->h == pi->h && pj->tau == pi->tau;
            for (int a = 0; a < b->D; ++a) same = same && pj->N[a] == pi->N[a];
            if (same) owner[i] = j;
        }
        if (owner[i] < 0) return SDF_ERR_INVALID_ARG;  // cannot happen for a batch built by sdf_batch_create
    }
    // tune each owner on its own problem (padded sizes and tile schedule) ...
    for (int i = 0; i < n; ++i) {
        if (owner[i] != i) continue;
        int rt, rf, fv;
        sdf_status s = sdf_plan_autotune(b->plans[i], K[i], points[i], weights ? weights[i] : nullptr, reps, &rt,
                                         &rf, &fv);
        if (s != SDF_OK) return s;
    }
    // ... and give its sizes, spectra and schedule to the problems that share them
    for (int i = 0; i < n; ++i) {
        if (owner[i] == i) continue;
        sdf_plan o = b->plans[owner[i]], pi = b->plans[i];
        bool sameM = true;
        for (int a = 0; a < b->D; ++a) sameM = sameM && o->M[a] == pi->M[a];
        if (!sameM) {
            sdf_status s = plan_repad(pi, o->M, o);
            if (s != SDF_OK) return s;
        }
        pi->tune_RT = o->tune_RT;
        pi->tune_RF = o->tune_RF;
        pi->tune_FV = o->tune_FV;
        pi->tune_EV = o->tune_EV;
    }
    // the captured graph is stale now: the next sdf_batch_execute captures anew
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    b->K.clear();
    b->ptrs.clear();
    return SDF_OK;
}

sdf_status sdf_batch_sync(sdf_batch b) {
    if (!b) return SDF_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return fail(e);
    sdf_status first = SDF_OK;
    for (auto p : b->plans) {
        sdf_status s = sdf_sync(p);
        if (s != SDF_OK && first == SDF_OK) first = s;
    }
    return first;
}

sdf_plan sdf_batch_plan(sdf_batch b, int i) {
    if (!b || i < 0 || i >= b->n) return nullptr;
    return b->plans[i];
}

void sdf_batch_destroy(sdf_batch b) {
    if (!b) return;
    batch_free(b);
    delete b;
}

}  // extern "C"
