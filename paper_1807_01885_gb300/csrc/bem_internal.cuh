// Internal declarations shared by the CUDA translation units of libbem.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <utility>
#include <vector>

#include "bem.h"

namespace bem {

// ---------------------------------------------------------------------------
// complex arithmetic on float2 / double2
template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx = typename cplx_of<T>::type;

__host__ __device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }
__host__ __device__ __forceinline__ double2 mk(double x, double y) { return make_double2(x, y); }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
// float: the real and imaginary parts added by one packed two-wide instruction
// (.f32x2, sm_100 family): half the issue slots of the FFT butterflies' additions
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return mk(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { return mk(a.y, -a.x); }
template <typename C> __device__ __forceinline__ C cmul_pi(C a) { return mk(-a.y, a.x); }

// ---------------------------------------------------------------------------
// Layout constants.
// Spectrum (after the row pass), N >= 16: column-major, spec[j * N + r] for the
// frequencies j in [0, N] (each column contiguous for the column pass; the row
// passes move whole 32-byte groups of neighbouring rows through shared memory).
// N < 16 (the small-grid shared-memory kernels): column-block-major, for column
// block cb (TC consecutive frequencies) an N x TC row-major sub-array
//     spec[((cb * N) + r) * TC + tc],  j = cb * TC + tc,  cb in [0, N/TC],
// the last block holding only the Nyquist column j = N at tc = 0.  Both fit in
// (N/TC + 1) N TC complex values.
constexpr int TC = 4;
constexpr int NTHREADS = 256;
constexpr int MAX_LOGN = 11;   // N <= 2048

// Device-side scalar state of a solve (double throughout).
struct SolveState {
  double d;          // current depth
  double gbar;       // mean gap over the contact set (force control)
  double G, Gold;    // sum of squared gaps, previous value
  double beta;       // CG direction factor
  double flag;       // 1 = conjugate step allowed, 0 = steepest descent restart
  double tau;        // step length
  double rbar;       // mean of K t over the contact set (force control)
  double res;        // relative residual
  double sum_p;      // sum of pressures after the update
  double scale;      // pending load-control rescale of p (1 = none)
  double uscale;     // rms displacement over the contact set (noise thresholds)
  double res_replaced; // residual at the last replacement of the recursive gap by the true one
  double pscale;     // mean pressure over the contact set
  double target;     // F under force control
  double delta2;     // delta^2
  double tol;
  double rr, rr_new, b2;       // linear CG (adhesive inner solve)
  double alpha;
  double qbar;       // mean of K s over the contact area (adhesive force control)
  double lin_rbar;   // mean of the residual over the area: its rounding drift (adhesive force control)
  double lin_shift;  // uniform pressure added on the area to carry the force (adhesive force control)
  double sig_c;      // Eq. (12) detachment stress
  uint64_t mask_hash;
  int n_c;           // contact cells at the start of the iteration
  int n_neg, n_ol;   // projected cells, re-activated cells
  int n_add, n_detach;
  int iter;
  int done;          // 1 once converged
  int refresh;       // 1: recompute u = K p before the next step
  int status;        // bem_status raised on the device (BEM_ENAN)
  int control;
  int max_iter;
  int matvecs;
  int mv_p_on;       // gate of the refresh product u = K p (1 = run)
  int mv_t_on;       // gate of the search-direction product (1 = run, i.e. not done)
  int replace;       // 1: recompute the gap from u = K p before the next iteration
  int x_clear;       // 1: this iteration consumed x (its correction ran), so the update rewrites x from 0
  int restart_next;  // 1: the last direction was not a descent direction (no step taken): restart
  int loops;         // bodies of the device-side iteration loop executed
  int max_loops;     // bound on them (iteration limit / chunk + 2)
};

// Workspace owned by a kernel handle.
// Guard zones: every large workspace array is allocated with kGuard bytes of the
// pattern kGuardByte before and after it (the payload keeps the allocation's 256-byte
// alignment); bem_check_guards counts the guard bytes that no longer hold it.
constexpr size_t kGuard = 256;
constexpr unsigned char kGuardByte = 0xB5;
constexpr int kMaxGuarded = 16;
struct GuardRec {
  unsigned char* base = nullptr;   // start of the allocation (leading guard)
  size_t bytes = 0;                // payload size
};

struct Workspace {
  void* spec = nullptr;      // (N/TC + 1) * N * TC complex
  void* table = nullptr;     // K^/M^2 in the path precision: N >= 16 (N+1) rows of N+4 (row j = column j), else blocked
  double* table64 = nullptr; // (N+1)^2 doubles, unscaled, row-major
  void* tw = nullptr;        // M complex: e^{-2 pi i k / M}
  void* twr = nullptr;       // stage twiddles of the length-N register FFT (rows)
  void* twc = nullptr;       // stage twiddles of the length-2N register FFT (columns)
  void* twpc = nullptr;      // float path: broadcast stage twiddles of the paired column FFT (4N float4)
  void* vec = nullptr;       // solver vectors: p, g, t, r, u, f, x (N*N each)
  uint8_t* mask = nullptr;   // N*N contact mask (adhesive), plus a second copy; PK: contact set {p > 0}
  double* partials = nullptr;// per-block partial sums
  unsigned int* ticket = nullptr;
  SolveState* state = nullptr;
  SolveState* state_host = nullptr;   // pinned mirror
  double* aux_host = nullptr;         // pinned: final sums [0..4], non-finite count [7]
  cudaEvent_t done_ev = nullptr;      // batch rounds: state copied back
  void* stage_in = nullptr;  // staging for host arguments (N*N)
  void* stage_out = nullptr;
  GuardRec guards[kMaxGuarded];      // the guarded allocations (all of the arrays above but ticket and state)
  int n_guards = 0;
  unsigned long long* guard_bad = nullptr;   // device counter of bem_check_guards
};

}  // namespace bem

struct bem_kernel_s {
  bem_kernel_desc desc;
  int N, M, logN;
  int prec;       // BEM_FP64 / BEM_FP32
  size_t elem;    // sizeof(real)
  int dev;
  int n_layers = 0;    // > 0: coating stack of bem_make_kernel_layers (replaces h, E1, nu1)
  bem_layer layers[BEM_MAX_LAYERS];
  int col_radix_alt;   // 1: radix 8 for the float column pass (bem_set_radix, bem_autotune)
  int row_radix_alt;   // 1: radix 8 for the float row passes (bem_set_radix, bem_autotune)
  bem::Workspace ws;
  // per-pass CUDA-event timing (bem_set_pass_timing): pending (start, end) pairs,
  // harvested into totals at synchronisation points
  struct PassTiming {
    int on = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[3], pool;
    double ms[3] = {0, 0, 0};
    long long n[3] = {0, 0, 0};
  };
  mutable PassTiming timing;
  // captured iteration chunks (replayed by solves on this handle): the constrained
  // CG of non-adhesive solves and the fixed-area linear CG of adhesive ones
  struct Graphs {
    int warm = 0;                      // one chunk ran plainly (kernel attributes are set)
    cudaGraphExec_t pk_exec = nullptr;
    long long pk_nodes = 0;            // kernel nodes in pk_exec (launch accounting)
    int lin_warm = 0;
    cudaGraphExec_t lin_exec = nullptr;
    long long lin_nodes = 0;
    const void* lin_mask = nullptr;    // contact mask the linear chunk was captured with
    // the whole constrained-CG iteration as one graph: a conditional 'while' node whose
    // body is one chunk plus the loop control (device-side loop, no host round trip)
    cudaGraphExec_t loop_exec = nullptr;
    long long loop_nodes = 0;          // kernel nodes per body execution
  };
  Graphs graphs;
  uint64_t serial = 0;  // identity of the handle's captured kernels (new on creation and radix change)
};

namespace bem {
// True on the first call for the current device (devices 0..63) with this flag:
// one-time per-device setup such as kernel attributes, which are per device.
// Concurrent first calls may both see true; the setup they guard is idempotent.
inline bool first_on_device(std::atomic<unsigned long long>& seen) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  return (seen.fetch_or(bit) & bit) == 0;
}

void set_error(const std::string& msg);
// number of kernel launches issued by the library (for launch accounting)
void note_launches(long long n);

// Programmatic dependent launch along the iteration's kernel chain: a kernel launched
// with launch_pdl may be scheduled while its predecessor's last blocks still run.
// Every such kernel first waits for its predecessor grid (its results are then
// visible) and then lets its own successor be scheduled, so each kernel starts only
// after all earlier ones completed; what overlaps is the launch and block set-up with
// the predecessor's tail.  Outside a programmatic launch both are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}
long long launches();
// adds the durations of completed timed passes of k to its totals (host sync point)
void harvest_pass_timing(const bem_kernel_s* k);
bem_status cuda_fail(cudaError_t e, const char* what);
// api.cu: a library-owned stream of the current device used only to capture graphs
cudaStream_t capture_stream();
// api.cu: a fresh identity for a handle's captured kernels
uint64_t next_serial();
// api.cu: BEM_OK when the description is valid, else BEM_EINVAL with a message
bem_status check_desc(const bem_kernel_desc* d);
// the open-plane operator's body is homogeneous: h = INFINITY (E1, nu1), h = 0 (E2,
// nu2) or both materials equal; *E, *nu receive its modulus and Poisson ratio
inline bool open_plane_homogeneous(const bem_kernel_desc& d, double* E = nullptr, double* nu = nullptr) {
  double e = 0.0, n = 0.0;
  bool ok = true;
  if (d.h == INFINITY) { e = d.E1; n = d.nu1; }
  else if (d.h == 0.0 || (d.E1 == d.E2 && d.nu1 == d.nu2)) { e = d.E2; n = d.nu2; }
  else ok = false;
  if (ok && !(e > 0.0 && e < INFINITY)) ok = false;
  if (E != nullptr) *E = e;
  if (nu != nullptr) *nu = n;
  return ok;
}

// matvec.cu
bem_status build_table(bem_kernel_s* k, cudaStream_t s);
template <typename T>
void launch_matvec(const bem_kernel_s* k, const T* p, T* u, cudaStream_t s, const int* skip_flag);
// one pass of the product (0 = rows forward, 1 = columns, 2 = rows inverse)
template <typename T>
void launch_pass(const bem_kernel_s* k, int pass, const T* p, T* u, cudaStream_t s);
size_t spec_bytes(const bem_kernel_s* k);
// matvec_f32.cu / matvec_f64.cu (N >= 16)
template <typename T>
void reg_pass(const bem_kernel_s* k, int which, const T* p, T* u, cudaStream_t s, const int* skip);
template <typename T>
void reg_twiddles(const bem_kernel_s* k, cudaStream_t s);
template <typename T>
void reg_prepare(const bem_kernel_s* k);
// matvec.cu: sets the one-time kernel attributes of the product's passes for k
// (what the first plain launch would set), so that a graph capture can follow
template <typename T>
void prepare_passes(const bem_kernel_s* k);
int stage_tw_count(int logl);
// float4 records of the paired FFT's stage twiddles for length 2^logl (upper bound)
int pair_tw_count(int logl);
size_t table_bytes(const bem_kernel_s* k);

// solve.cu
bem_status solve_contact(bem_kernel_s* k, const bem_problem* prob, void* p_out, bem_result* res,
                         cudaStream_t s);
}  // namespace bem

#define BEM_CUDA_TRY(call)                                     \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return bem::cuda_fail(e_, #call);   \
  } while (0)
