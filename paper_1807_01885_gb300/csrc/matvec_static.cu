// u = K p without any device allocation, for callers that cannot allocate.
//
// Some callers are not allowed to call cudaMalloc: code that runs inside a
// memory-capped or pre-reserved allocator (the memory pool of a host framework
// that must not be bypassed), code in a real-time loop where an allocation could
// block or fail, and plug-ins that are handed device buffers but no allocation
// rights.  bem_matvec_static serves them: the caller passes the operator
// parameters, the input p and the output u, and every intermediate the product
// needs (the double compliance table and its scaled copy, the twiddle tables and
// the half spectrum between the FFT passes) lives in one fixed array in device
// memory, `g_static_scratch` below, sized for grids up to BEM_STATIC_MAX_N.
//
// The array is a file-scope __device__ variable, so every GPU on which the library
// is loaded holds it until the process exits.  Host code cannot use the array's
// name as a device address; the first call on each device asks the runtime for the
// address (cudaGetSymbolAddress, with that device current) and keeps it.  All calls
// share the array and it keeps the last call's contents: every call rewrites all of
// it that it reads, so nothing has to be cleared between calls, but calls that
// overlap on the GPU (on different streams, or from several threads) race on it.
#include <string>

#include "bem_internal.cuh"

namespace bem {
namespace {

constexpr size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// Byte layout of the scratch for a grid of N cells per side (float path).
struct StaticLayout {
  size_t spec, table64, table, tw, twr, twc, twpc, total;
  explicit StaticLayout(int N) {
    const size_t c = 2 * sizeof(float);
    const size_t blocked = (size_t)(N / TC + 1) * (N + 1) * TC, square = (size_t)(N + 1) * (N + 4);
    size_t off = 0;
    spec = off;
    off += round256((size_t)(N / TC + 1) * N * TC * c);
    table64 = off;
    off += round256((size_t)(N + 1) * (N + 1) * sizeof(double));
    table = off;
    off += round256((blocked > square ? blocked : square) * sizeof(float));
    tw = off;
    off += round256((size_t)2 * N * c);
    twr = off;
    off += round256((size_t)2 * N * c);
    twc = off;
    off += round256((size_t)4 * N * c);
    twpc = off;
    off += round256((size_t)4 * N * 4 * sizeof(float));
    total = off;
  }
};

constexpr size_t kStaticBytes = 1400 * 1024;   // >= StaticLayout(BEM_STATIC_MAX_N).total

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices] = {nullptr};

bem_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("bem_matvec_static: device index out of range");
    return BEM_EUNSUPPORTED;
  }
  if (g_scratch_ptr[dev] == nullptr) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_static_scratch)");
    g_scratch_ptr[dev] = ptr;
  }
  *out = g_scratch_ptr[dev];
  return BEM_OK;
}

// True for device (or managed) memory that belongs to device dev: the scratch array
// and the stream the kernels run on are those of the current device, so an array of
// another GPU would be read and written through peer access or fault.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace
}  // namespace bem

using namespace bem;

extern "C" bem_status bem_matvec_static(const bem_kernel_desc* desc, const float* p, float* u, void* cuda_stream) {
  if (desc == nullptr || p == nullptr || u == nullptr) {
    set_error("bem_matvec_static: NULL argument");
    return BEM_EINVAL;
  }
  // the same operator checks as bem_make_kernel, then the limits of this entry point
  bem_status st = check_desc(desc);
  if (st != BEM_OK) return st;
  const int N = desc->N;
  if (N > BEM_STATIC_MAX_N) {
    set_error("bem_matvec_static: N must be a power of two in [4, " + std::to_string(BEM_STATIC_MAX_N) +
              "] (the fixed scratch array is sized for that); use bem_make_kernel/bem_matvec for larger grids");
    return BEM_EINVAL;
  }
  if (desc->precision != BEM_FP32) {
    set_error("bem_matvec_static: only precision BEM_FP32 is available");
    return BEM_EINVAL;
  }
  if (desc->op_kind != BEM_OP_PERIODIC) {
    set_error("bem_matvec_static: only the periodic operator (op_kind BEM_OP_PERIODIC) is available");
    return BEM_EINVAL;
  }
  if (((uintptr_t)p & 15) != 0 || ((uintptr_t)u & 15) != 0) {
    set_error("bem_matvec_static: p and u must be 16-byte aligned");
    return BEM_EINVAL;
  }
  int dev = 0;
  BEM_CUDA_TRY(cudaGetDevice(&dev));
  if (!on_device(p, dev) || !on_device(u, dev)) {
    set_error("bem_matvec_static: p and u must be device arrays of the current device (host arrays would need "
              "a staging allocation)");
    return BEM_EINVAL;
  }
  void* base = nullptr;
  st = scratch_address(dev, &base);
  if (st != BEM_OK) return st;
  const StaticLayout lay(N);
  if (lay.total > kStaticBytes) {
    set_error("bem_matvec_static: internal scratch layout exceeds the fixed array");
    return BEM_EUNSUPPORTED;
  }
  // A handle on the stack whose workspace points into the fixed array; only the
  // fields the table build and the three passes read are set.
  bem_kernel_s k{};
  k.desc = *desc;
  k.N = N;
  k.M = 2 * N;
  k.logN = 0;
  while ((1 << k.logN) < N) ++k.logN;
  k.prec = BEM_FP32;
  k.elem = sizeof(float);
  k.dev = dev;
  unsigned char* b = (unsigned char*)base;
  k.ws.spec = b + lay.spec;
  k.ws.table64 = (double*)(b + lay.table64);
  k.ws.table = b + lay.table;
  k.ws.tw = b + lay.tw;
  k.ws.twr = b + lay.twr;
  k.ws.twc = b + lay.twc;
  k.ws.twpc = b + lay.twpc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  st = build_table(&k, s);
  if (st != BEM_OK) return st;
  launch_matvec<float>(&k, p, u, s, nullptr);
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}
