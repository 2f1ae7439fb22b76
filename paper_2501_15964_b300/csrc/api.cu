// Context, error reporting, scratch memory and scans for libccm.
#include "ccm_internal.cuh"

namespace ccm {

static thread_local std::string g_last_error = "no error";

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file,
            line);
  return e == cudaErrorMemoryAllocation ? CCM_ERR_OOM : CCM_ERR_CUDA;
}

int ws_get(Ctx* c, Slot s, size_t bytes, void** out) {
  bytes = bytes ? bytes : 16;
  if (c->slot_size[s] < bytes) {
    if (c->slot_ptr[s]) {
      CCM_CUDA(cudaFree(c->slot_ptr[s]));
      c->slot_ptr[s] = nullptr;
      c->slot_size[s] = 0;
    }
    size_t want = (size_t)round_up((int64_t)bytes, 256);
    cudaError_t e = cudaMalloc(&c->slot_ptr[s], want);
    if (e != cudaSuccess) {
      c->slot_ptr[s] = nullptr;
      set_error("scratch allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
      return CCM_ERR_OOM;
    }
    c->slot_size[s] = want;
  }
  *out = c->slot_ptr[s];
  return CCM_OK;
}

int host_scalars(Ctx* c, size_t bytes, void** out) {
  if (c->host_pinned_size < bytes) {
    if (c->host_pinned) CCM_CUDA(cudaFreeHost(c->host_pinned));
    c->host_pinned = nullptr;
    CCM_CUDA(cudaMallocHost(&c->host_pinned, bytes));
    c->host_pinned_size = bytes;
  }
  *out = c->host_pinned;
  return CCM_OK;
}

// ------------------------------------------------------------------ scan
// Exclusive prefix sum of int64 values: tiles of 1024 scanned in shared
// memory, tile totals scanned recursively, then added back.
static constexpr int SCAN_TILE = 1024;

__global__ void k_scan_tiles(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                             int64_t* __restrict__ tile_sums, int64_t n) {
  __shared__ int64_t sh[SCAN_TILE];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int t = threadIdx.x;
  int64_t v = (base + t < n) ? in[base + t] : 0;
  sh[t] = v;
  __syncthreads();
  for (int o = 1; o < SCAN_TILE; o <<= 1) {
    int64_t add = (t >= o) ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += add;
    __syncthreads();
  }
  if (base + t < n) out[base + t] = sh[t] - v;
  if (t == SCAN_TILE - 1) tile_sums[blockIdx.x] = sh[t];
}

__global__ void k_scan_add(int64_t* __restrict__ out, const int64_t* __restrict__ offs,
                           int64_t n) {
  int64_t i = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x;
  if (i < n) out[i] += offs[blockIdx.x];
}

static int scan_rec(Ctx* c, const int64_t* in, int64_t* out, int64_t n, int level,
                    cudaStream_t s) {
  int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (level >= 6) {
    set_error("scan too deep");
    return CCM_ERR_INVALID_ARG;
  }
  void* buf;
  // two buffers per level: tile sums and their scan
  CCM_TRY(ws_get(c, (Slot)(S_SCRATCH0 + 2 * level), (size_t)tiles * 8, &buf));
  int64_t* sums = (int64_t*)buf;
  CCM_TRY(ws_get(c, (Slot)(S_SCRATCH0 + 2 * level + 1), (size_t)tiles * 8, &buf));
  int64_t* sums_scan = (int64_t*)buf;
  k_scan_tiles<<<(unsigned)tiles, SCAN_TILE, 0, s>>>(in, out, sums, n);
  CCM_COUNT(c);
  CCM_CUDA(cudaGetLastError());
  if (tiles > 1) {
    CCM_TRY(scan_rec(c, sums, sums_scan, tiles, level + 1, s));
    k_scan_add<<<(unsigned)tiles, SCAN_TILE, 0, s>>>(out, sums_scan, n);
    CCM_COUNT(c);
    CCM_CUDA(cudaGetLastError());
  }
  return CCM_OK;
}

__global__ void k_scan_total(const int64_t* in, const int64_t* out, int64_t n, int64_t* tot) {
  *tot = n > 0 ? out[n - 1] + in[n - 1] : 0;
}

// Exclusive scan; if total_host != NULL the total is copied back (synchronising s).
// Uses scratch slots S_SCRATCH0.. (callers must not hold those across this call).
int scan_exclusive_i64(Ctx* c, const int64_t* in, int64_t* out, int64_t n, int64_t* total_host,
                       cudaStream_t s) {
  if (n <= 0) {
    if (total_host) *total_host = 0;
    return CCM_OK;
  }
  CCM_TRY(scan_rec(c, in, out, n, 0, s));
  if (total_host) {
    void* hp;
    CCM_TRY(host_scalars(c, 64, &hp));
    void* dtot;
    CCM_TRY(ws_get(c, S_SCRATCH7, 16, &dtot));
    k_scan_total<<<1, 1, 0, s>>>(in, out, n, (int64_t*)dtot);
    CCM_COUNT(c);
    CCM_CUDA(cudaGetLastError());
    CCM_CUDA(cudaMemcpyAsync(hp, dtot, 8, cudaMemcpyDeviceToHost, s));
    CCM_CUDA(cudaStreamSynchronize(s));
    *total_host = *(int64_t*)hp;
  }
  return CCM_OK;
}

}  // namespace ccm

using namespace ccm;

extern "C" {

struct ccm_ctx {
  Ctx c;
};

const char* ccm_last_error(void) { return ccm::g_last_error.c_str(); }

int32_t ccm_max_dim(void) { return 1024; }

void ccm_default_options(ccm_options* o) {
  if (!o) return;
  o->sigma0 = 1.0;
  o->sigma_max = 0.0;  // automatic: resolve_sigma_max()
  o->max_outer = 200;
  o->max_newton = 50;
  o->max_cg = 500;
  o->precision = CCM_PREC_MIXED;
  o->engine = CCM_ENGINE_AUTO;
  o->profile = 0;
  o->relabel = 1;
  o->autotune = 1;
  o->coarse = 0;
  o->X0 = nullptr;
  o->U0 = nullptr;
}

int ccm_create(ccm_ctx** out, int device) {
  if (!out) {
    set_error("ccm_create: out is NULL");
    return CCM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  int count = 0;
  CCM_CUDA(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) {
    set_error("ccm_create: device %d out of range (%d devices)", device, count);
    return CCM_ERR_INVALID_ARG;
  }
  CCM_CUDA(cudaSetDevice(device));
  ccm_ctx* x = new ccm_ctx();
  x->c.device = device;
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) {
    delete x;
    return cuda_fail(e, "cudaGetDeviceProperties", __FILE__, __LINE__);
  }
  x->c.num_sms = prop.multiProcessorCount;
  x->c.l2_bytes = prop.l2CacheSize;
  *out = x;
  return CCM_OK;
}

void ccm_destroy(ccm_ctx* x) {
  if (!x) return;
  cudaSetDevice(x->c.device);
  for (int s = 0; s < S_COUNT; ++s)
    if (x->c.slot_ptr[s]) cudaFree(x->c.slot_ptr[s]);
  if (x->c.host_pinned) cudaFreeHost(x->c.host_pinned);
  for (auto ev : x->c.ev_pool) cudaEventDestroy(ev);
  if (x->c.copy_event) cudaEventDestroy(x->c.copy_event);
  if (x->c.copy_stream) cudaStreamDestroy(x->c.copy_stream);
  delete x;
}

int64_t ccm_launch_count(ccm_ctx* x) { return x ? x->c.launches : 0; }

int ccm_last_profile(ccm_ctx* x, ccm_profile* out) {
  if (!x || !out) {
    set_error("ccm_last_profile: NULL argument");
    return CCM_ERR_INVALID_ARG;
  }
  *out = x->c.last_profile;
  return CCM_OK;
}

int ccm_last_graph_info(ccm_ctx* x, ccm_graph_info* out) {
  if (!x || !out) {
    set_error("ccm_last_graph_info: NULL argument");
    return CCM_ERR_INVALID_ARG;
  }
  *out = x->c.last_graph;
  return CCM_OK;
}

}  // extern "C"

namespace ccm {
Ctx* ctx_of(ccm_ctx* x) { return x ? &x->c : nullptr; }
}  // namespace ccm
