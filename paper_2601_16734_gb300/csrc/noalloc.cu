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
// call on each device, with that device current, asks the runtime for the
// device address once (cudaGetSymbolAddress) and caches it.  That first call
// should therefore come before any stream capture.
//
// All calls share the one array and leave their intermediates in it: two
// calls whose kernels overlap on the GPU (different streams, or different
// host threads) race and corrupt each other's results.  Serialise them.
// Every scratch word a call reads is written earlier by the same call, so no
// clearing is needed.
#include <mutex>

#include "contract.cuh"

#define SEEMPS_NOALLOC_SCRATCH_BYTES (32u << 20)  // 32 MiB
#define SEEMPS_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[SEEMPS_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_setup_mutex;
void* g_scratch_addr[SEEMPS_NOALLOC_MAX_DEVICES] = {nullptr};

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
  // scratch layout of the FP64 apply (see heff_plan): 512 bytes of status
  // words, the (D_l d^2) x (d^2 D_r) mixing matrix, T1 and T2
  const size_t need = 512 + align256((size_t)(Dl * d * d) * (d * d * Dr) * 8) +
                      align256((size_t)(chil * Dl * d * d * chir) * 8) +
                      align256((size_t)(chil * d * d * Dr * chir) * 8) + 256;
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
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= SEEMPS_NOALLOC_MAX_DEVICES) {
    write_error(errbuf, errbuf_len, "heff_apply_noalloc: no usable current device");
    return SEEMPS_ERR_CUDA;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        write_error(errbuf, errbuf_len, "heff_apply_noalloc: cudaGetSymbolAddress failed");
        return SEEMPS_ERR_CUDA;
      }
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
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
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
    ctx.sm_count = sms;
  HeffPlan plan;
  seemps_status st = heff_plan(&ctx, dims, L, W1, W2, R, SEEMPS_FP64, &plan);
  if (st == SEEMPS_OK) st = heff_run(&ctx, &plan, theta, y);
  if (st != SEEMPS_OK) write_error(errbuf, errbuf_len, ctx.err);
  return st;
}
