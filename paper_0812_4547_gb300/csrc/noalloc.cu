// noalloc.cu -- a sketch entry point that never allocates memory.
//
// Some callers cannot allocate device memory at the point where they need a
// sketch: code running while a memory pool is frozen or fully reserved by a
// framework, real-time loops that must not call into the allocator (it can
// synchronise the device or fail under fragmentation), and hosts that hand
// out only pre-registered buffers.  rnnls_sketch_noalloc serves them: the
// caller passes the inputs and outputs, and all scratch space (sampled rows
// when no idx buffer is given, the combine plan, the per-chunk-range partial
// sums) comes from one fixed array compiled into this library.
//
// The array is a file-scope __device__ variable: every GPU on which the
// entry point has been called holds kNoAllocScratchBytes of it until the
// process exits (with lazy module loading the driver reserves it, with this
// file's kernels, at the first call on a device).  Host code cannot use the
// array's name as a device address; the set-up asks the runtime for the
// current device's address (cudaGetSymbolAddress) and remembers it together
// with the unique ID of the context it belongs to.  When the current context
// changes (cudaDeviceReset and a new primary context, or a context the
// caller made current) the next call repeats the set-up, since the array
// can then sit at another address.
#include <cuda.h>  // CUcontext (the two driver calls are fetched at run time)
#include <math.h>

#include <mutex>

#include "kernels.h"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;  // 8 MiB per device
constexpr int64_t kNoAllocMaxRows = 16384;                  // largest r accepted
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

typedef CUresult (*ctx_get_current_fn)(CUcontext *);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long *);

std::mutex g_setup_mutex;
struct device_setup {
  unsigned long long ctx_id;  // unique ID of the context the address belongs to
  void *addr;                 // device address of g_noalloc_scratch in that context
  int num_sms;
};
device_setup g_setup[kMaxDevices];

// The unique ID of the current context (cuCtxGetId: never reused within the
// process, unlike the context handle), or 0 when it cannot be read.
unsigned long long current_context_id() {
  static ctx_get_current_fn get_current = nullptr;
  static ctx_get_id_fn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<ctx_get_current_fn>(p);
    else
      cudaGetLastError();
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<ctx_get_id_fn>(p);
    else
      cudaGetLastError();
  });
  if (!get_current || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// With device `dev` current: the device address of the scratch array and the
// SM count, looked up once per device and again whenever the current
// context is not the one the stored address was taken in.
int setup_device(int dev, void **addr, int *num_sms) {
  if (dev < 0 || dev >= kMaxDevices) return RNNLS_EUNSUPPORTED;
  unsigned long long id = current_context_id();  // 0 also when no context is bound to the thread yet
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  device_setup &su = g_setup[dev];
  if (id == 0 || su.ctx_id != id || !su.addr) {
    // the lookup binds the runtime's context of `dev` to this thread if needed
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return RNNLS_ECUDA;
    }
    id = current_context_id();
    if (id == 0) return RNNLS_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return RNNLS_ECUDA;
    }
    su.ctx_id = id;
    su.addr = p;
    su.num_sms = sms;
  }
  *addr = su.addr;
  *num_sms = su.num_sms;
  return RNNLS_OK;
}

}  // namespace

extern "C" int rnnls_sketch_noalloc(void *stream, const float *A, int64_t lda, const float *b, int64_t n_raw,
                                    int64_t d, int64_t r, uint64_t seed, uint64_t instance, float *SA, int64_t ldsa,
                                    float *Sb, int32_t *idx) {
  using namespace rnnls;
  if (!A || !b || !SA || !Sb) return RNNLS_EINVAL;
  if (n_raw < 1 || d < 1 || r < 1 || lda < n_raw || ldsa < r) return RNNLS_EINVAL;
  if (n_raw > ((int64_t)1 << 28) || d > (1 << 20) || r > kNoAllocMaxRows) return RNNLS_EUNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return RNNLS_ECUDA;
  }
  void *scratch = nullptr;
  int num_sms = 0;
  int st = setup_device(dev, &scratch, &num_sms);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // scratch layout: [sampled rows when idx is null][plan + partial sums]
  char *base = (char *)scratch;
  size_t used = 0;
  int32_t *rows = idx;
  if (!rows) {
    rows = (int32_t *)base;
    used = align_up((size_t)r * sizeof(int32_t), 256);
  }
  const int L = log2_ceil64(n_raw);
  st = launch_sample_iid(s, seed, instance, L, r, rows);
  if (st) return st;
  sketch_args_f32 a;
  a.A = A;
  a.lda = lda;
  a.b = b;
  a.n_raw = n_raw;
  a.d = (int)d;
  a.L = L;
  a.r = r;
  a.d_count = nullptr;
  a.seed = seed;
  a.inst = instance;
  a.scale = (float)(1.0 / sqrt((double)r));
  a.SA = SA;
  a.ldsa = ldsa;
  a.Sb = Sb;
  a.ldb = n_raw;
  a.nb = 1;
  a.ldsb = ldsa;
  a.chunk0 = 0;
  a.idx = rows;
  a.gen_iid = 0;
  return sketch_f32_scratch(s, a, num_sms, base + used, kNoAllocScratchBytes - used);
}
