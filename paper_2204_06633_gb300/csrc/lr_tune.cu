// CUDA-graph capture of the batched response and the tile autotuner.
//
// Graph: an MCMC step re-evaluates the same batch shapes with new strain values; capturing the
// batched call (tile-table kernel + persistent fused kernel) once and replaying it removes the
// host-side launch work from every step.  The captured pointers are fixed: the caller rewrites
// the inputs in place between replays.
//
// Autotuner: the fastest tile size depends on the order, the precision and the GPU; it is found
// by timing the fused kernel on a synthetic series for a few candidate tiles, and cached in a
// small text file keyed by (GPU name, precision, order, generation, length bucket).
#include <cuda_runtime.h>
#include <sys/stat.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lr_launch.h"
#include "lr_planview.h"

struct lr_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    // the graph's own batch tables (tile prefix sums [S+1], then the sources' sky frames [S+1]):
    // the plan's batch tables are re-allocated when a later call brings a larger batch, so a
    // replay must not depend on them
    int64_t *tables;
};

namespace {

std::string cache_path()
{
    const char *e = std::getenv("LR_AUTOTUNE_CACHE");
    if (e && *e) return e;
    const char *home = std::getenv("HOME");
    return std::string(home ? home : "/tmp") + "/.cache/lisaresp_autotune.txt";
}

std::string tune_key(const lr::PlanView &v, int generation, int64_t n)
{
    cudaDeviceProp prop;
    std::memset(&prop, 0, sizeof(prop));
    cudaGetDeviceProperties(&prop, v.device);
    std::string name = prop.name;
    for (char &c : name)
        if (c == ' ') c = '_';
    int bucket = n > 0 ? (int)std::floor(std::log2((double)n)) : 0;
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s|p%d|o%d|g%d|b%d", name.c_str(), v.precision, v.order, generation, bucket);
    return buf;
}

int cache_lookup(const std::string &key)
{
    FILE *f = std::fopen(cache_path().c_str(), "r");
    if (!f) return 0;
    char k[256];
    int tile = 0, found = 0;
    double ms;
    while (std::fscanf(f, "%255s %d %lf", k, &tile, &ms) == 3)
        if (key == k) found = tile;  // the last entry for a key wins
    std::fclose(f);
    return found;
}

void cache_store(const std::string &key, int tile, double ms)
{
    std::string path = cache_path();
    const size_t cut = path.find_last_of('/');
    if (cut != std::string::npos && cut > 0) mkdir(path.substr(0, cut).c_str(), 0755);  // best effort
    FILE *f = std::fopen(path.c_str(), "a");
    if (!f) return;
    std::fprintf(f, "%s %d %.6f\n", key.c_str(), tile, ms);
    std::fclose(f);
}

std::vector<int> tile_candidates(const lr::PlanView &v)
{
    std::vector<int> cand;
    if (v.precision == LR_MIXED) {
        // the largest tile the shared-memory arrays hold, and smaller ones
        const int tmax = lr::mx_max_tile(v.base.HL, v.base.HR, v.base.lproj_b, v.order + 1);
        cand.push_back(tmax);
        for (int t : {256, 192, 128})
            if (t < tmax) cand.push_back(t);
    } else {
        for (int t : {256, 384, 512, 768, 1024}) cand.push_back(t);
    }
    return cand;
}

// Largest |exp(i w eps) - sum_j w_j(eps) exp(i w j)| over eps in [0, 1) (129 points) for the
// centered Lagrange read of degree p (nodes j = -(p-1)/2 .. (p+1)/2, weights by direct products):
// the read error of a unit complex sinusoid of w radians per sample.
double lagrange_sinusoid_error(int p, double w)
{
    const int h = (p - 1) / 2, T = p + 1;
    double worst = 0.0;
    for (int k = 0; k <= 128; ++k) {
        const double eps = k / 128.0;
        double re = 0.0, im = 0.0;
        for (int a = 0; a < T; ++a) {
            const int ja = a - h;
            double wa = 1.0;
            for (int b = 0; b < T; ++b)
                if (b != a) wa *= (eps - (double)(b - h)) / (double)(ja - (b - h));
            re += wa * std::cos(w * ja);
            im += wa * std::sin(w * ja);
        }
        const double dr = std::cos(w * eps) - re, di = std::sin(w * eps) - im;
        worst = std::max(worst, std::sqrt(dr * dr + di * di));
    }
    return worst;
}

}  // namespace

extern "C" {

LR_API int lr_choose_order(double f_dt, double tol, int *order)
{
    if (!order || !(f_dt >= 0.0) || !(f_dt < 0.5) || !(tol > 0.0) || !std::isfinite(tol)) return LR_ERR_INVALID_ARG;
    const double w = 2.0 * 3.14159265358979323846 * f_dt;
    for (int p = 1; p <= 63; p += 2) {
        if (!lr::order_supported(p)) continue;
        if (lagrange_sinusoid_error(p, w) <= tol) {
            *order = p;
            return LR_OK;
        }
    }
    return LR_ERR_RANGE;
}

LR_API int lr_response_batched_graph(lr_plan *plan, int64_t S, const int64_t *h_off, const int64_t *out_off,
                                     const double *t0_h, const lr_sky *sky, const double *hp, const double *hc,
                                     double *xyz, lr_graph **out)
{
    if (!plan || !out) return LR_ERR_INVALID_ARG;
    *out = nullptr;
    if (S < 1) return LR_ERR_INVALID_ARG;
    if (S > (int64_t)1 << 24) return LR_ERR_RANGE;
    if (!h_off || !out_off || !t0_h || !sky || !hp || !hc || !xyz) return LR_ERR_INVALID_ARG;
    lr::PlanView v;
    int st = lr::plan_view(plan, &v);
    if (st) return st;
    lr_graph *g = new (std::nothrow) lr_graph();
    if (!g) return LR_ERR_OOM;
    g->graph = nullptr;
    g->exec = nullptr;
    g->tables = nullptr;
    // the graph's tables are allocated before the capture (nothing may allocate during it)
    cudaError_t e = lr::dev_malloc((void **)&g->tables, (sizeof(int64_t) + sizeof(lr::SkyConst)) * (size_t)(S + 1));
    if (e != cudaSuccess) {
        delete g;
        return e == cudaErrorMemoryAllocation ? LR_ERR_OOM : lr::plan_cuda_fail(plan, e);
    }
    lr::SkyConst *skyc =
        v.precision == LR_MIXED ? reinterpret_cast<lr::SkyConst *>(g->tables + (S + 1)) : nullptr;
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        lr::FwdParams P = v.base;
        int le = lr::launch_batch_tables(out_off, sky, S, P.tile, g->tables, skyc, P.err, cs);
        P.src.skyc = skyc;
        P.src.h_off = h_off;
        P.src.out_off = out_off;
        P.src.t0h = t0_h;
        P.src.sky = sky;
        P.src.tile_off = g->tables;
        P.src.S = S;
        P.hp = hp;
        P.hc = hc;
        P.out = xyz;
        P.total_tiles = -1;
        if (!le) le = lr::launch_forward(v.precision, lr::KIND_FUSED, v.order, P, v.threads, v.sms, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &g->graph);
        e = le ? (cudaError_t)le : e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        cudaFree(g->tables);
        delete g;
        return lr::plan_cuda_fail(plan, e);
    }
    *out = g;
    return LR_OK;
}

LR_API int lr_graph_launch(lr_graph *graph, void *stream)
{
    if (!graph || !graph->exec) return LR_ERR_INVALID_ARG;
    return cudaGraphLaunch(graph->exec, (cudaStream_t)stream) == cudaSuccess ? LR_OK : LR_ERR_CUDA;
}

LR_API int lr_graph_destroy(lr_graph *graph)
{
    if (!graph) return LR_ERR_INVALID_ARG;
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    if (graph->tables) cudaFree(graph->tables);
    delete graph;
    return LR_OK;
}

LR_API int lr_plan_autotune(lr_plan *plan, int64_t n_samples, int use_cache, void *stream, int *tile_out)
{
    if (!plan || !tile_out) return LR_ERR_INVALID_ARG;
    if (n_samples < 1024 || n_samples > ((int64_t)1 << 28)) return LR_ERR_RANGE;
    lr::PlanView v;
    int st = lr::plan_view(plan, &v);
    if (st) return st;
    const int generation = v.base.q_terms == 3 ? 1 : 2;
    const std::string key = tune_key(v, generation, n_samples);
    if (use_cache) {
        int t = cache_lookup(key);
        if (t > 0 && lr::plan_set_tile(plan, t) == LR_OK) {
            *tile_out = t;
            return LR_OK;
        }
    }
    std::vector<int> cand = tile_candidates(v);
    // synthetic single-source problem with all the input margins the plan needs
    const int64_t left = v.base.sig_b + v.base.lproj_b + v.order / 2 + 4, right = v.base.sig_b + v.order / 2 + 4;
    const int64_t nh = n_samples + left + right;
    double *h = nullptr, *out = nullptr;
    cudaError_t e = lr::dev_malloc((void **)&h, sizeof(double) * (size_t)nh);
    if (e == cudaSuccess) e = lr::dev_malloc((void **)&out, sizeof(double) * 3 * (size_t)n_samples);
    if (e == cudaSuccess) e = cudaMemsetAsync(h, 0, sizeof(double) * (size_t)nh, (cudaStream_t)stream);
    cudaEvent_t a = nullptr, b = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const int tile0 = v.base.tile;
    int best = tile0;
    double best_ms = 1e300;
    // time a plan-sized single-source call: build the launch as lr_response would
    for (size_t i = 0; e == cudaSuccess && i < cand.size(); ++i) {
        if (lr::plan_set_tile(plan, cand[i]) != LR_OK) continue;
        lr::PlanView w;
        lr::plan_view(plan, &w);
        lr::FwdParams P = w.base;
        P.src.n1 = n_samples;
        P.src.nh1 = nh;
        P.src.t0h1 = P.t0 - (double)left * P.dt;
        P.src.sky1 = lr_sky{1.0, 0.3, 0.4};
        P.src.skyc1 = lr::make_sky(P.src.sky1);
        P.hp = h;
        P.hc = h;
        P.out = out;
        P.total_tiles = (n_samples + P.tile - 1) / P.tile;
        int le = lr::launch_forward(w.precision, lr::KIND_FUSED, w.order, P, w.threads, w.sms, stream);
        if (le) continue;  // e.g. the tile needs more shared memory than a CTA may have
        cudaEventRecord(a, (cudaStream_t)stream);
        for (int r = 0; r < 3; ++r) lr::launch_forward(w.precision, lr::KIND_FUSED, w.order, P, w.threads, w.sms, stream);
        cudaEventRecord(b, (cudaStream_t)stream);
        e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && ms / 3.0 < best_ms) {
            best_ms = ms / 3.0;
            best = cand[i];
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (h) cudaFree(h);
    if (out) cudaFree(out);
    lr::plan_set_tile(plan, best_ms < 1e300 ? best : tile0);
    if (e != cudaSuccess) return lr::plan_cuda_fail(plan, e);
    if (best_ms < 1e300 && use_cache) cache_store(key, best, best_ms);
    *tile_out = best_ms < 1e300 ? best : tile0;
    return LR_OK;
}

LR_API int lr_plan_autotune_batch(lr_plan *plan, int64_t S, const int64_t *lengths, int use_cache, void *stream,
                                  int *tile_out)
{
    if (!plan || !lengths || !tile_out) return LR_ERR_INVALID_ARG;
    if (S < 1 || S > ((int64_t)1 << 24)) return LR_ERR_RANGE;
    lr::PlanView v;
    int st = lr::plan_view(plan, &v);
    if (st) return st;
    // the batch's length distribution: up to 48 quantiles, scaled so the synthetic batch holds at
    // most 2^24 outputs (the tile choice depends on the mix of lengths, not on the batch size)
    std::vector<int64_t> sorted(lengths, lengths + S);
    for (int64_t x : sorted)
        if (x < 0) return LR_ERR_INVALID_ARG;
    std::sort(sorted.begin(), sorted.end());
    const int64_t k = std::min<int64_t>(S, 48);
    std::vector<int64_t> lens((size_t)k);
    double tot = 0.0;
    for (int64_t i = 0; i < k; ++i) {
        lens[(size_t)i] = sorted[(size_t)((2 * i + 1) * S / (2 * k))];
        tot += (double)lens[(size_t)i];
    }
    if (tot < 1.0) return LR_ERR_RANGE;
    const double scale = std::min(1.0, (double)(1 << 24) / tot);
    const int generation = v.base.q_terms == 3 ? 1 : 2;
    char sig[160];
    std::snprintf(sig, sizeof(sig), "|batch%lld_%.0f_%.0f_%.0f", (long long)S, std::log2((double)sorted[(size_t)(S / 10)] + 1),
                  std::log2((double)sorted[(size_t)(S / 2)] + 1), std::log2((double)sorted[(size_t)(9 * S / 10)] + 1));
    const std::string key = tune_key(v, generation, 0) + sig;
    if (use_cache) {
        int t = cache_lookup(key);
        if (t > 0 && lr::plan_set_tile(plan, t) == LR_OK) {
            *tile_out = t;
            return LR_OK;
        }
    }
    const int64_t left = v.base.sig_b + v.base.lproj_b + v.order / 2 + 4, right = v.base.sig_b + v.order / 2 + 4;
    std::vector<int64_t> hoff((size_t)k + 1, 0), ooff((size_t)k + 1, 0);
    std::vector<double> t0h((size_t)k);
    std::vector<lr_sky> sky((size_t)k);
    for (int64_t i = 0; i < k; ++i) {
        const int64_t n = std::max<int64_t>(1, (int64_t)(scale * (double)lens[(size_t)i]));
        ooff[(size_t)i + 1] = ooff[(size_t)i] + n;
        hoff[(size_t)i + 1] = hoff[(size_t)i] + n + left + right;
        t0h[(size_t)i] = v.base.t0 - (double)left * v.base.dt;
        sky[(size_t)i] = lr_sky{0.3 + 0.1 * (double)i, 0.2, 0.4};
    }
    const int64_t nh = hoff[(size_t)k], no = ooff[(size_t)k];
    double *h = nullptr, *out = nullptr, *d_t0h = nullptr;
    int64_t *d_off = nullptr, *tables = nullptr;
    lr_sky *d_sky = nullptr;
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e = lr::dev_malloc((void **)&h, sizeof(double) * (size_t)nh);
    if (e == cudaSuccess) e = lr::dev_malloc((void **)&out, sizeof(double) * 3 * (size_t)no);
    if (e == cudaSuccess) e = lr::dev_malloc((void **)&d_off, sizeof(int64_t) * 2 * (size_t)(k + 1));
    if (e == cudaSuccess) e = lr::dev_malloc((void **)&d_t0h, sizeof(double) * (size_t)k);
    if (e == cudaSuccess) e = lr::dev_malloc((void **)&d_sky, sizeof(lr_sky) * (size_t)k);
    if (e == cudaSuccess) e = lr::dev_malloc((void **)&tables, (sizeof(int64_t) + sizeof(lr::SkyConst)) * (size_t)(k + 1));
    if (e == cudaSuccess) e = cudaMemsetAsync(h, 0, sizeof(double) * (size_t)nh, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, hoff.data(), sizeof(int64_t) * (size_t)(k + 1), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_off + k + 1, ooff.data(), sizeof(int64_t) * (size_t)(k + 1), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_t0h, t0h.data(), sizeof(double) * (size_t)k, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_sky, sky.data(), sizeof(lr_sky) * (size_t)k, cudaMemcpyHostToDevice, cs);
    cudaEvent_t a = nullptr, b = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const int tile0 = v.base.tile;
    int best = tile0;
    double best_ms = 1e300;
    const std::vector<int> cand = tile_candidates(v);
    lr::SkyConst *skyc = v.precision == LR_MIXED ? reinterpret_cast<lr::SkyConst *>(tables + k + 1) : nullptr;
    for (size_t i = 0; e == cudaSuccess && i < cand.size(); ++i) {
        if (lr::plan_set_tile(plan, cand[i]) != LR_OK) continue;
        lr::PlanView w;
        lr::plan_view(plan, &w);
        lr::FwdParams P = w.base;
        P.src.skyc = skyc;
        P.src.h_off = d_off;
        P.src.out_off = d_off + k + 1;
        P.src.t0h = d_t0h;
        P.src.sky = d_sky;
        P.src.tile_off = tables;
        P.src.S = k;
        P.hp = h;
        P.hc = h;
        P.out = out;
        P.total_tiles = -1;
        // one batched call = the batch tables and the persistent fused kernel, as lr_response_batched
        auto call = [&]() {
            int le = lr::launch_batch_tables(P.src.out_off, d_sky, k, P.tile, tables, skyc, P.err, cs);
            return le ? le : lr::launch_forward(w.precision, lr::KIND_FUSED, w.order, P, w.threads, w.sms, cs);
        };
        if (call()) continue;
        cudaEventRecord(a, cs);
        for (int r = 0; r < 3; ++r) call();
        cudaEventRecord(b, cs);
        e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && ms / 3.0 < best_ms) {
            best_ms = ms / 3.0;
            best = cand[i];
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    for (void *p : {(void *)h, (void *)out, (void *)d_t0h, (void *)d_off, (void *)tables, (void *)d_sky})
        if (p) cudaFree(p);
    lr::plan_set_tile(plan, best_ms < 1e300 ? best : tile0);
    if (e != cudaSuccess) return lr::plan_cuda_fail(plan, e);
    if (best_ms < 1e300 && use_cache) cache_store(key, best, best_ms);
    *tile_out = best_ms < 1e300 ? best : tile0;
    return LR_OK;
}

}  // extern "C"
