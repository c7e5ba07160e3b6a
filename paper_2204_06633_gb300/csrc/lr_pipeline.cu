// Batched forward response on host buffers, pipelined in chunks of sources.
//
// lr_response_batched works on device-resident batches.  A caller whose strain and results live
// in host memory would otherwise copy the whole batch in, compute, and copy the whole result
// out, one after the other.  Here the batch is cut into chunks of whole sources and three
// streams overlap the copy-in of chunk c+1, the fused kernel on chunk c and the copy-out of chunk
// c-1, with two device slots used in turn.  Ordering between the streams is by events:
//   copy-in of a slot waits for the kernel that last read that slot's inputs;
//   the kernel waits for its copy-in and for the copy-out of the slot's previous results;
//   copy-out waits for the kernel.
// The host refills a slot's pinned staging (rebased offsets, start times, sky) only after the
// copy-in that last read it has completed.  The call returns when every result is on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "lr_launch.h"
#include "lr_pipeline.h"
#include "lr_planview.h"

namespace lr {

namespace {

// output samples per chunk (a chunk holds at least one whole source); LR_PIPELINE_CHUNK_OUTPUTS
// overrides it (tests use small chunks to run many of them)
int64_t chunk_outputs()
{
    const char *s = std::getenv("LR_PIPELINE_CHUNK_OUTPUTS");
    if (s) {
        const long long v = std::atoll(s);
        if (v >= 1) return (int64_t)v;
    }
    return int64_t(1) << 25;
}

struct PipeSlot {
    double *h = nullptr;        // h+ [cap_h] then hx [cap_h]
    double *xyz = nullptr;      // [3 cap_n]
    int64_t *tab = nullptr;     // tile table [cap_s + 1] then sky frames [cap_s + 1]
    int64_t *hoff = nullptr;    // rebased [cap_s + 1]
    int64_t *ooff = nullptr;    // rebased [cap_s + 1]
    double *t0h = nullptr;      // [cap_s]
    lr_sky *sky = nullptr;      // [cap_s]
    char *pin = nullptr;        // pinned staging of hoff, ooff, t0h, sky
    cudaEvent_t in = nullptr, run = nullptr, out = nullptr;
};

}  // namespace

struct PipeWork {
    int64_t cap_h = 0, cap_n = 0, cap_s = 0;
    cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
    PipeSlot slot[2];
};

static void free_slot(PipeSlot &q)
{
    if (q.h) cudaFree(q.h);
    if (q.xyz) cudaFree(q.xyz);
    if (q.tab) cudaFree(q.tab);
    if (q.hoff) cudaFree(q.hoff);
    if (q.pin) cudaFreeHost(q.pin);
    if (q.in) cudaEventDestroy(q.in);
    if (q.run) cudaEventDestroy(q.run);
    if (q.out) cudaEventDestroy(q.out);
    q = PipeSlot();
}

void pipe_free(PipeWork *w)
{
    if (!w) return;
    for (auto &q : w->slot) free_slot(q);
    if (w->s_in) cudaStreamDestroy(w->s_in);
    if (w->s_run) cudaStreamDestroy(w->s_run);
    if (w->s_out) cudaStreamDestroy(w->s_out);
    delete w;
}

// small per-slot arrays in one device allocation: hoff, ooff [cap_s + 1] each, t0h, sky [cap_s]
static size_t small_bytes(int64_t cap_s)
{
    return 2 * sizeof(int64_t) * (size_t)(cap_s + 1) + (sizeof(double) + sizeof(lr_sky)) * (size_t)cap_s;
}

// makes sure both slots hold a chunk of (nh, nn, ns); grows (re-allocates) when needed
static cudaError_t pipe_reserve(PipeWork &w, int64_t nh, int64_t nn, int64_t ns)
{
    if (nh <= w.cap_h && nn <= w.cap_n && ns <= w.cap_s && w.slot[0].h) return cudaSuccess;
    const int64_t ch = std::max(nh, w.cap_h), cn = std::max(nn, w.cap_n), cs = std::max(ns, w.cap_s);
    for (auto &q : w.slot) {
        free_slot(q);
        cudaError_t e = dev_malloc((void **)&q.h, sizeof(double) * 2 * (size_t)ch);
        if (e == cudaSuccess) e = dev_malloc((void **)&q.xyz, sizeof(double) * 3 * (size_t)cn);
        if (e == cudaSuccess) e = dev_malloc((void **)&q.tab, (sizeof(int64_t) + sizeof(SkyConst)) * (size_t)(cs + 1));
        if (e == cudaSuccess) e = dev_malloc((void **)&q.hoff, small_bytes(cs));
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&q.pin, small_bytes(cs), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q.in, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q.run, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q.out, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (auto &r : w.slot) free_slot(r);
            w.cap_h = w.cap_n = w.cap_s = 0;
            return e;
        }
        q.ooff = q.hoff + (cs + 1);
        q.t0h = reinterpret_cast<double *>(q.ooff + (cs + 1));
        q.sky = reinterpret_cast<lr_sky *>(q.t0h + cs);
    }
    w.cap_h = ch;
    w.cap_n = cn;
    w.cap_s = cs;
    return cudaSuccess;
}

}  // namespace lr

extern "C" LR_API int lr_response_batched_host(lr_plan *plan, int64_t S, const int64_t *h_off,
                                               const int64_t *out_off, const double *t0_h, const lr_sky *sky,
                                               const double *hp, const double *hc, double *xyz, void *stream)
{
    using namespace lr;
    if (!plan || !h_off || !out_off || !t0_h || !sky || !hp || !hc || !xyz) return LR_ERR_INVALID_ARG;
    if (S < 1) return LR_ERR_INVALID_ARG;
    if (S > (int64_t)1 << 24) return LR_ERR_RANGE;
    for (int64_t s = 0; s < S; ++s)
        if (h_off[s + 1] < h_off[s] || out_off[s + 1] < out_off[s]) return LR_ERR_INVALID_ARG;
    if (h_off[0] != 0 || out_off[0] != 0) return LR_ERR_INVALID_ARG;
    PlanView v;
    int st = plan_view(plan, &v);
    if (st) return st;
    // chunks of whole sources, about chunk_outputs() outputs each
    const int64_t target = chunk_outputs();
    std::vector<int64_t> cut{0};
    int64_t mh = 0, mn = 0, ms = 0;
    for (int64_t s = 0; s < S; ++s) {
        const int64_t c0 = cut.back();
        if (s + 1 == S || out_off[s + 1] - out_off[c0] >= target) {
            cut.push_back(s + 1);
            mh = std::max(mh, h_off[s + 1] - h_off[c0]);
            mn = std::max(mn, out_off[s + 1] - out_off[c0]);
            ms = std::max(ms, s + 1 - c0);
        }
    }
    PipeWork *&wp = plan_pipe(plan);
    if (!wp) {
        wp = new (std::nothrow) PipeWork();
        if (!wp) return LR_ERR_OOM;
        cudaError_t e = cudaStreamCreateWithFlags(&wp->s_in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&wp->s_run, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&wp->s_out, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            pipe_free(wp);
            wp = nullptr;
            return plan_cuda_fail(plan, e);
        }
    }
    PipeWork &w = *wp;
    cudaError_t e = pipe_reserve(w, std::max<int64_t>(mh, 1), std::max<int64_t>(mn, 1), ms);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LR_ERR_OOM : plan_cuda_fail(plan, e);
    // work already queued on the caller's stream comes first
    cudaEvent_t start = nullptr;
    e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(start, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(w.s_in, start, 0);
    const int nchunk = (int)cut.size() - 1;
    for (int c = 0; e == cudaSuccess && c < nchunk; ++c) {
        PipeSlot &q = w.slot[c & 1];
        const int64_t s0 = cut[c], s1 = cut[c + 1], ns = s1 - s0;
        const int64_t h0 = h_off[s0], nh = h_off[s1] - h0, o0 = out_off[s0], nn = out_off[s1] - o0;
        // staging: the copy-in that last read this slot's pinned buffer must be done
        e = cudaEventSynchronize(q.in);
        if (e != cudaSuccess) break;
        int64_t *ph = reinterpret_cast<int64_t *>(q.pin), *po = ph + (w.cap_s + 1);
        double *pt = reinterpret_cast<double *>(po + (w.cap_s + 1));
        lr_sky *pk = reinterpret_cast<lr_sky *>(pt + w.cap_s);
        for (int64_t i = 0; i <= ns; ++i) {
            ph[i] = h_off[s0 + i] - h0;
            po[i] = out_off[s0 + i] - o0;
        }
        std::memcpy(pt, t0_h + s0, sizeof(double) * (size_t)ns);
        std::memcpy(pk, sky + s0, sizeof(lr_sky) * (size_t)ns);
        // copy in, after the kernel that last read this slot
        e = cudaStreamWaitEvent(w.s_in, q.run, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(q.h, hp + h0, sizeof(double) * (size_t)nh, cudaMemcpyHostToDevice, w.s_in);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(q.h + w.cap_h, hc + h0, sizeof(double) * (size_t)nh, cudaMemcpyHostToDevice, w.s_in);
        if (e == cudaSuccess) e = cudaMemcpyAsync(q.hoff, q.pin, small_bytes(w.cap_s), cudaMemcpyHostToDevice, w.s_in);
        if (e == cudaSuccess) e = cudaEventRecord(q.in, w.s_in);
        // compute, after the copy-in and after the copy-out of this slot's previous results
        if (e == cudaSuccess) e = cudaStreamWaitEvent(w.s_run, q.in, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(w.s_run, q.out, 0);
        if (e != cudaSuccess) break;
        FwdParams P = v.base;
        SkyConst *skyc = v.precision == LR_MIXED ? reinterpret_cast<SkyConst *>(q.tab + (w.cap_s + 1)) : nullptr;
        int le = launch_batch_tables(q.ooff, q.sky, ns, P.tile, q.tab, skyc, P.err, w.s_run);
        if (!le) {
            P.src.skyc = skyc;
            P.src.h_off = q.hoff;
            P.src.out_off = q.ooff;
            P.src.t0h = q.t0h;
            P.src.sky = q.sky;
            P.src.tile_off = q.tab;
            P.src.S = ns;
            P.hp = q.h;
            P.hc = q.h + w.cap_h;
            P.out = q.xyz;
            P.total_tiles = -1;
            le = launch_forward(v.precision, KIND_FUSED, v.order, P, v.threads, v.sms, w.s_run);
        }
        if (le) {
            e = (cudaError_t)le;
            break;
        }
        e = cudaEventRecord(q.run, w.s_run);
        // copy out
        if (e == cudaSuccess) e = cudaStreamWaitEvent(w.s_out, q.run, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(xyz + 3 * o0, q.xyz, sizeof(double) * 3 * (size_t)nn, cudaMemcpyDeviceToHost, w.s_out);
        if (e == cudaSuccess) e = cudaEventRecord(q.out, w.s_out);
    }
    // every queued copy finishes before return, also after a failure
    cudaError_t e2 = cudaStreamSynchronize(w.s_out);
    cudaError_t e3 = cudaStreamSynchronize(w.s_run);
    cudaError_t e4 = cudaStreamSynchronize(w.s_in);
    if (start) cudaEventDestroy(start);
    if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : (e3 != cudaSuccess ? e3 : e4);
    return e == cudaSuccess ? LR_OK : plan_cuda_fail(plan, e);
}
