// Effective-operator apply (FP64) for callers that cannot allocate device
// memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not
// possible - a host application whose device memory is owned by another
// allocator that will not hand out a buffer, a plugin loaded into such a
// process, or a caller that must not trigger any allocation (and the
// implicit device synchronisation cudaFree can cause) inside a latency
// critical loop.  Every other entry point of this library needs a
// caller-allocated workspace; this one does not.
//
// How: the intermediates (the MPO mixing matrix and the two partial
// contractions) live in one file-scope __device__ array of
// SEEMPS_NOALLOC_SCRATCH_BYTES.  Every GPU that loads the library holds that
// array until the process exits.  Host code cannot use the array's name as a
// device address (in host code it names a host-side stand-in), so the first
// call in each CUDA context (the device's primary context, or one the caller
// created with the driver API), with that context current, asks the runtime
// for the array's device address once (cudaGetSymbolAddress) and caches it
// under the context's process-unique id (cuCtxGetId): an address is only
// valid in the context it was looked up in, and a context recreated after
// cudaDeviceReset gets a new id and a fresh lookup.  That first call should
// therefore come before any stream capture.  (If the driver entry points
// are missing, every call looks the address up again.)
//
// All calls share the one array and leave their intermediates in it: two
// calls whose kernels overlap on the GPU (different streams, or different
// host threads) race and corrupt each other's results.  Serialise them.
// Every scratch word a call reads is written earlier by the same call, so no
// clearing is needed.
#include <cuda.h>

#include <mutex>

#include "contract.cuh"

#define SEEMPS_NOALLOC_SCRATCH_BYTES (32u << 20)  // 32 MiB
#define SEEMPS_NOALLOC_MAX_CONTEXTS 64
// Largest accepted dimensions (checked before any size arithmetic, so that
// the scratch size below cannot overflow).
#define SEEMPS_NOALLOC_MAX_CHI (1 << 20)
#define SEEMPS_NOALLOC_MAX_SMALL (1 << 10)  // d and the MPO bonds

static __device__ __align__(256) unsigned char g_noalloc_scratch[SEEMPS_NOALLOC_SCRATCH_BYTES];

namespace {

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

std::mutex g_setup_mutex;
struct ScratchEntry {
  unsigned long long ctx_id;
  void* addr;
};
ScratchEntry g_scratch[SEEMPS_NOALLOC_MAX_CONTEXTS];
int g_scratch_n = 0;
bool g_driver_loaded = false;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Driver entry points for the current context's id (loaded once, under the mutex).
void load_driver_entries() {
  if (g_driver_loaded) return;
  g_driver_loaded = true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess && fn)
    g_ctx_get_current = (CtxGetCurrentFn)fn;
  fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess && fn)
    g_ctx_get_id = (CtxGetIdFn)fn;
}

// Device address of the scratch array in the current context: cached per
// context id, looked up (cudaGetSymbolAddress) on the first call in a context.
cudaError_t scratch_address(void** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  load_driver_entries();
  unsigned long long id = 0;
  bool have_id = false;
  CUcontext cur = nullptr;
  if (g_ctx_get_current && g_ctx_get_id && g_ctx_get_current(&cur) == CUDA_SUCCESS && cur &&
      g_ctx_get_id(cur, &id) == CUDA_SUCCESS)
    have_id = true;
  if (have_id) {
    for (int i = 0; i < g_scratch_n; ++i)
      if (g_scratch[i].ctx_id == id) {
        *out = g_scratch[i].addr;
        return cudaSuccess;
      }
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  if (!p) return cudaErrorInvalidSymbol;
  if (have_id) {
    const int slot = g_scratch_n < SEEMPS_NOALLOC_MAX_CONTEXTS ? g_scratch_n++ : (int)(id % SEEMPS_NOALLOC_MAX_CONTEXTS);
    g_scratch[slot].ctx_id = id;
    g_scratch[slot].addr = p;
  }
  *out = p;
  return cudaSuccess;
}

void write_error(char* buf, size_t len, const char* msg) {
  if (buf && len) {
    snprintf(buf, len, "%s", msg);
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" seemps_status seemps_heff_apply_noalloc(const seemps_pair_dims* dims, const double* L,
                                                   const double* W1, const double* W2,
                                                   const double* R, const double* theta, double* y,
                                                   void* stream, char* errbuf, size_t errbuf_len) {
  if (!dims || !L || !W1 || !W2 || !R || !theta || !y) {
    write_error(errbuf, errbuf_len, "heff_apply_noalloc: null argument");
    return SEEMPS_ERR_INVALID;
  }
  if (theta == y) {
    write_error(errbuf, errbuf_len, "heff_apply_noalloc: y may not alias theta");
    return SEEMPS_ERR_INVALID;
  }
  const ll chil = dims->chi_l, chir = dims->chi_r, d = dims->d;
  const ll Dl = dims->D_l, Dm = dims->D_m, Dr = dims->D_r;
  if (chil <= 0 || chir <= 0 || d <= 0 || Dl <= 0 || Dm <= 0 || Dr <= 0) {
    write_error(errbuf, errbuf_len, "heff_apply_noalloc: non-positive dimension");
    return SEEMPS_ERR_INVALID;
  }
  // bound every dimension first; even then a size such as chi^2 d^2 D can
  // reach 2^70 bytes, so the sizes are formed one factor at a time with
  // overflow checks before they are compared with the scratch size
  if (chil > SEEMPS_NOALLOC_MAX_CHI || chir > SEEMPS_NOALLOC_MAX_CHI || d > SEEMPS_NOALLOC_MAX_SMALL ||
      Dl > SEEMPS_NOALLOC_MAX_SMALL || Dm > SEEMPS_NOALLOC_MAX_SMALL || Dr > SEEMPS_NOALLOC_MAX_SMALL) {
    write_error(errbuf, errbuf_len, "heff_apply_noalloc: dimension out of range (chi <= 2^20, d, D <= 2^10)");
    return SEEMPS_ERR_INVALID;
  }
  size_t wmat = 0, t1 = 0, t2 = 0;
  bool ovf = false;
  auto mul = [&ovf](size_t a, size_t b) {
    size_t r = 0;
    ovf |= __builtin_mul_overflow(a, b, &r);
    return r;
  };
  wmat = mul(mul(mul(mul((size_t)Dl, (size_t)(d * d)), (size_t)(d * d)), (size_t)Dr), 8);
  t1 = mul(mul(mul(mul((size_t)chil, (size_t)Dl), (size_t)(d * d)), (size_t)chir), 8);
  t2 = mul(mul(mul(mul((size_t)chil, (size_t)(d * d)), (size_t)Dr), (size_t)chir), 8);
  if (ovf || wmat > SEEMPS_NOALLOC_SCRATCH_BYTES || t1 > SEEMPS_NOALLOC_SCRATCH_BYTES ||
      t2 > SEEMPS_NOALLOC_SCRATCH_BYTES) {
    write_error(errbuf, errbuf_len, "heff_apply_noalloc: these sizes need more scratch than the maximum of "
                                    "32 MiB (chi_l * chi_r * D * d^2 * 16 bytes must stay below it)");
    return SEEMPS_ERR_WORKSPACE;
  }
  // scratch layout of the FP64 apply (see heff_plan): 512 bytes of status
  // words, the (D_l d^2) x (d^2 D_r) mixing matrix, T1 and T2
  const size_t need = 512 + align256(wmat) + align256(t1) + align256(t2) + 256;
  if (need > SEEMPS_NOALLOC_SCRATCH_BYTES) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "heff_apply_noalloc: these sizes need %zu bytes of scratch, the maximum is %u "
             "(chi_l * chi_r * D * d^2 * 16 bytes must stay below it)",
             need, (unsigned)SEEMPS_NOALLOC_SCRATCH_BYTES);
    write_error(errbuf, errbuf_len, msg);
    return SEEMPS_ERR_WORKSPACE;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    write_error(errbuf, errbuf_len, "heff_apply_noalloc: no usable current device");
    return SEEMPS_ERR_CUDA;
  }
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess || !base) {
    write_error(errbuf, errbuf_len, "heff_apply_noalloc: cudaGetSymbolAddress failed");
    return SEEMPS_ERR_CUDA;
  }
  // A context on the stack that carves from the static scratch instead of a
  // caller workspace; no allocation of any kind.
  seemps_ctx ctx;
  memset(&ctx, 0, sizeof ctx);
  ctx.device = dev;
  ctx.stream = (cudaStream_t)stream;
  ctx.ws = (char*)base;
  ctx.ws_bytes = SEEMPS_NOALLOC_SCRATCH_BYTES;
  ctx.d_status = (int*)base;
  ctx.d_scalars = (double*)((char*)base + 256);
  ctx.ws_top = 512;
  ctx.sm_count = 1;
  ctx.wait_clocks = SEEMPS_WAIT_CLOCKS;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
    ctx.sm_count = sms;
  HeffPlan plan;
  seemps_status st = heff_plan(&ctx, dims, L, W1, W2, R, SEEMPS_FP64, &plan);
  if (st == SEEMPS_OK) st = heff_run(&ctx, &plan, theta, y);
  if (st != SEEMPS_OK) write_error(errbuf, errbuf_len, ctx.err);
  return st;
}
