// Batched forward response that allocates no device memory.
//
// lr_response_batched keeps its per-batch tile table in memory the plan allocates with
// cudaMalloc on first use (and re-allocates when a larger batch arrives).  Some callers may
// not allocate at that point: a sampler or serving process that has handed its whole device
// memory budget to its own allocator up front, or one that cannot afford the device-wide
// synchronisation a cudaMalloc / cudaFree implies in the middle of a run.  This variant keeps
// the tile table in a fixed file-scope device array instead, so the call itself allocates
// nothing; the price is a fixed capacity (LR_NOALLOC_MAX_SOURCES sources) held by every GPU
// that loads the library, for the life of the process.
#include <cuda_runtime.h>

#include <mutex>

#include "lr_launch.h"
#include "lr_planview.h"

namespace {

constexpr int64_t kMaxSources = LR_NOALLOC_MAX_SOURCES;
constexpr int kMaxDevices = 64;

// the tile table: prefix sums of tiles per source, [S+1] entries, and the sources' sky frames
// [S] (mixed precision), rewritten in full by every call
static __device__ __align__(256) int64_t g_tile_table[kMaxSources + 1];
static __device__ __align__(256) lr::SkyConst g_sky_table[kMaxSources];

// device addresses of g_tile_table and g_sky_table on each device, looked up once per device
int64_t *g_table_addr[kMaxDevices];
lr::SkyConst *g_sky_addr[kMaxDevices];
std::mutex g_table_mutex;

// In host code g_tile_table and g_sky_table name host-side stand-ins, not device memory: their
// device addresses come from cudaGetSymbolAddress, taken once per device with that device current.
int table_address(int device, int64_t **out, lr::SkyConst **sky_out)
{
    if (device < 0 || device >= kMaxDevices) return (int)cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_table_mutex);
    if (!g_table_addr[device]) {
        int prev = -1;
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) return (int)e;
        if (prev != device) {
            e = cudaSetDevice(device);
            if (e != cudaSuccess) return (int)e;
        }
        void *p = nullptr, *q = nullptr;
        e = cudaGetSymbolAddress(&p, g_tile_table);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_sky_table);
        if (prev != device) {
            cudaError_t e2 = cudaSetDevice(prev);
            if (e == cudaSuccess) e = e2;
        }
        if (e != cudaSuccess) return (int)e;
        g_table_addr[device] = static_cast<int64_t *>(p);
        g_sky_addr[device] = static_cast<lr::SkyConst *>(q);
    }
    *out = g_table_addr[device];
    *sky_out = g_sky_addr[device];
    return 0;
}

}  // namespace

namespace lr {
// Called by lr_ctx_create with `device` current: looks up the arrays' device addresses now, which
// also makes the CUDA runtime load this file's module (and allocate the arrays) during set-up
// rather than inside a caller's first allocation-free call.
int noalloc_setup(int device)
{
    int64_t *table = nullptr;
    SkyConst *sky = nullptr;
    return table_address(device, &table, &sky);
}
}  // namespace lr

extern "C" LR_API int lr_response_batched_noalloc(lr_plan *plan, int64_t S, const int64_t *h_off,
                                                  const int64_t *out_off, const double *t0_h, const lr_sky *sky,
                                                  const double *hp, const double *hc, double *xyz, void *stream)
{
    if (!plan || !h_off || !out_off || !t0_h || !sky || !hp || !hc || !xyz) return LR_ERR_INVALID_ARG;
    if (S < 1) return LR_ERR_INVALID_ARG;
    if (S > kMaxSources) return LR_ERR_RANGE;
    lr::PlanView v;
    int st = lr::plan_view(plan, &v);
    if (st) return st;
    int64_t *table = nullptr;
    lr::SkyConst *skytab = nullptr;
    int e = table_address(v.device, &table, &skytab);
    if (e) return lr::plan_cuda_fail(plan, e);
    lr::FwdParams P = v.base;
    // every entry of the tables the launch reads is written first by these kernels
    lr::SkyConst *skyc = v.precision == LR_MIXED ? skytab : nullptr;
    e = lr::launch_batch_tables(out_off, sky, S, P.tile, table, skyc, P.err, stream);
    if (e) return lr::plan_cuda_fail(plan, e);
    P.src.skyc = skyc;
    P.src.h_off = h_off;
    P.src.out_off = out_off;
    P.src.t0h = t0_h;
    P.src.sky = sky;
    P.src.tile_off = table;
    P.src.S = S;
    P.hp = hp;
    P.hc = hc;
    P.out = xyz;
    P.total_tiles = -1;
    e = lr::launch_forward(v.precision, lr::KIND_FUSED, v.order, P, v.threads, v.sms, stream);
    return e ? lr::plan_cuda_fail(plan, e) : LR_OK;
}
