// Internal declarations shared by the libvie translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <utility>

#include "../../include/vie.h"

namespace vie {

// ---------------------------------------------------------------------------
// error reporting (thread-local message behind vie_last_error)
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

#define VIE_CUDA_TRY(expr)                                                    \
  do {                                                                        \
    cudaError_t e__ = (expr);                                                 \
    if (e__ != cudaSuccess) {                                                 \
      ::vie::set_error("%s:%d: %s failed: %s", __FILE__, __LINE__, #expr,     \
                       cudaGetErrorString(e__));                              \
      return e__ == cudaErrorMemoryAllocation ? VIE_ERR_OOM : VIE_ERR_CUDA;   \
    }                                                                         \
  } while (0)

#define VIE_LAUNCH_CHECK()                                                    \
  do {                                                                        \
    cudaError_t e__ = cudaGetLastError();                                     \
    if (e__ != cudaSuccess) {                                                 \
      ::vie::set_error("%s:%d: kernel launch failed: %s", __FILE__, __LINE__, \
                       cudaGetErrorString(e__));                              \
      return VIE_ERR_CUDA;                                                    \
    }                                                                         \
  } while (0)

// ---------------------------------------------------------------------------
// complex helpers on float2 / double2
// ---------------------------------------------------------------------------
template <typename R> struct cplx_t;
template <> struct cplx_t<float> { typedef float2 type; };
template <> struct cplx_t<double> { typedef double2 type; };

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename V> __host__ __device__ __forceinline__ V add(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename V> __host__ __device__ __forceinline__ V sub(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename V> __host__ __device__ __forceinline__ V mul(V a, V b) {
  V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <typename V> __host__ __device__ __forceinline__ V mulc(V a, V b) {
  V r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
template <typename V, typename R> __host__ __device__ __forceinline__ V scale(V a, R s) { V r; r.x = a.x * s; r.y = a.y * s; return r; }
// -i * a  and  +i * a
template <typename V> __host__ __device__ __forceinline__ V mul_mi(V a) { V r; r.x = a.y; r.y = -a.x; return r; }
template <typename V> __host__ __device__ __forceinline__ V mul_pi(V a) { V r; r.x = -a.y; r.y = a.x; return r; }

// ---------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialisation attribute may start before the previous kernel in the
// stream has finished.  It may read immutable plan data before pdl_wait(),
// but must call pdl_wait() before it reads anything an earlier kernel writes
// or writes anything at all.  pdl_launch_dependents() lets the next kernel
// start launching.  Both are no-ops for ordinary launches.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Launch with programmatic stream serialisation.
template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------------------
// FFT plans for one axis
// ---------------------------------------------------------------------------
constexpr int kMaxStages = 16;

struct AxisPlan {
  int len = 0;
  int nstages = 0;
  int radix[kMaxStages] = {0};
  float2* tw32 = nullptr;   // device, len entries: exp(-2 pi i k / len)
  double2* tw64 = nullptr;
};

// Radix list passed by value to kernels.
struct Radices {
  int len;
  int nstages;
  int r[kMaxStages];
};

inline Radices radices_of(const AxisPlan& a) {
  Radices r;
  r.len = a.len;
  r.nstages = a.nstages;
  for (int i = 0; i < kMaxStages; ++i) r.r[i] = a.radix[i];
  return r;
}

bool factor_length(int len, AxisPlan* out);   // radices from {4, 2, 3, 5}
bool factor_length_any(int len, AxisPlan* out);   // 4, 2, 3, 5, then larger primes (generic stages)
void x4_factors(int mx, int* l1, int* l2);    // compiled four-step split of Mx, or (0, 0)
void x3_factors(int mx, int* l1, int* l2, int* l3);   // compiled three-factor split of Mx, or zeros
int smooth_size_at_least(int n);               // smallest 5-smooth >= n

// ---------------------------------------------------------------------------
// the plan
// ---------------------------------------------------------------------------
}  // namespace vie

struct vie_plan {
  int n[3];
  int m[3];
  int kf[3];                  // folded (octant) spectrum extents m/2 + 1
  double h, k0, eps_bg, kappa;
  int device;
  vie::AxisPlan ax[3];
  // FP64 Toeplitz octant [6][nz][ny][nx]
  double2* toeplitz = nullptr;
  // folded spectra, pre-scaled by 1/(Mx My Mz): layout [kx'][c][kz'][ky']
  double2* ghat64 = nullptr;
  float2* ghat32 = nullptr;
  // contrast M per voxel [z][y][x]
  double2* M64 = nullptr;
  float2* M32 = nullptr;
  double2* chi64 = nullptr;
  // matvec workspace: 3*ny*nz lines x Mx spectra, sized for complex128
  void* work = nullptr;
  size_t work_bytes = 0;
  size_t device_bytes = 0;
  double setup_ms = 0.0;
  int* shared_refs = nullptr; // plans made by vie_plan_clone share entries, spectra and twiddles
  void* krylov = nullptr;     // solver workspace (vie::KrylovWork), created on first solve
  void* precond = nullptr;    // preconditioner state (learned or block-circulant), if set
  void* host_stage = nullptr; // device copies of b and x for solves on host buffers (2 x 3N complex128)
  size_t host_stage_bytes = 0;
  // JM-VIE (Sec. 3; allocated by vie_set_permeability)
  double2* curl = nullptr;    // FP64 octant of C_a, [3][nz][ny][nx]
  double2* chat64 = nullptr;  // folded curl spectra, [kx'][a][kz'][ky'], pre-scaled by 1/(Mx My Mz)
  float2* chat32 = nullptr;
  double2* Mjm64 = nullptr;   // 6N contrast: M_eps on the three electric, M_mu on the three magnetic components
  float2* Mjm32 = nullptr;
  double2* chimu64 = nullptr; // chi_mu = mu_r - 1 per voxel
  void* jm_work = nullptr;    // 6 ny nz Mx complex128
  int jm_gen = -1;            // contrast generation the 6N contrast was built from
  int contrast_gen = 0;       // incremented whenever the contrast is set
  int x_lpb = 0;              // forward x pass: > 0 four-step with that many lines per block,
                              // < 0 three-factor with -x_lpb lines per block, 0 heuristic
  int x_lpb_inv = 0;          // the same for the inverse x pass
  double tune_ms = 0.0;       // VIE_PLAN_AUTOTUNE host time
  int tune_candidates = 0;
};

namespace vie {

// GB300 streaming multiprocessors (grid sizing of the x passes)
constexpr int kSMs = 152;
// Five lines per x-pass block when that gives one block per SM where four
// lines would give more (the 600 x 23 x 11 guide: 759 lines, 152 blocks of
// five against 190 of four, 38 SMs then running two).  Compiled for the
// complex64 x passes with the line length fixed at 600.
inline bool x_lines_five(long NL, int count) {
  return (NL + 4) / 5 * count <= kSMs && (NL + 3) / 4 * count > kSMs;
}

vie_status compute_toeplitz(vie_plan* p, cudaStream_t s);
vie_status compute_curl(vie_plan* p, cudaStream_t s);     // C_a entries and folded spectra (JM-VIE)
// JM-VIE operator y = u - M (T u) on 6N vectors (u_e, u_m) of dtype; mode
// MODE_OPERATOR or MODE_RHS (then x is the 3N electric source current).
vie_status jm_matvec_impl(vie_plan* p, const void* x, void* y, int dtype, int mode, cudaStream_t s);
vie_status compute_spectrum(vie_plan* p, cudaStream_t s);
// `work` holds work_bytes; beyond the 3 ny nz Mx spectra of the x passes it
// may hold the y-pass buffer of the split pass B (pass_b_split_elems).
vie_status matvec_impl(vie_plan* p, const void* x, void* y, int dtype, int mode,
                       void* work, size_t work_bytes, cudaStream_t s);
// Complex values of the split pass B's buffer (Mx My 3 nz) when a plane of
// this shape takes it, else 0.
size_t pass_b_split_elems(int ny, int nz, int Mx, int My, int Mz);
// Looks up the static workspace of vie_matvec_static_scratch on the current
// device (loads its module there); plan creation calls it.
vie_status static_scratch_prepare();

// MODE_PLAIN (x-pass kernels run along y inside pass B): inverse FFT and
// crop only, no contrast epilogue.
enum { MODE_OPERATOR = 0, MODE_RHS = 1, MODE_PLAIN = 2 };

// Right preconditioner z = P(v) on vectors of type dtype (3 N complex).
typedef vie_status (*vie_precond_fn)(void* ctx, int dtype, const void* v, void* z, cudaStream_t s);

void free_krylov(vie_plan* p);
void free_precond(vie_plan* p);
vie_status precond_get(vie_plan* p, vie_precond_fn* fn, void** ctx);
int precond_fallback_flag(vie_plan* p, int clear);   // non-finite network output seen
int precond_is_learned(const vie_plan* p);            // the plan's preconditioner is a network
vie_status circulant_apply(vie_circulant* c, int dtype, const void* v, void* z, cudaStream_t s);
const vie_plan* circulant_plan(const vie_circulant* c);

// Operator application for `count` plans of one shape (same n and m);
// x[i], y[i] are device vectors of dtype; each plan's own workspace is used.
// live (optional): per plan a device flag read when the passes run; plans
// whose flag is 0 are skipped (y untouched).
vie_status matvec_group(vie_plan* const* plans, int count, const void* const* x, void* const* y, int dtype,
                        int mode, cudaStream_t s, const int* const* live = nullptr);
// jm != 0: the JM-VIE (6N unknowns per problem, jm_matvec_impl as operator).
vie_status solve_batch_impl(vie_plan* const* plans, int count, const double2* const* b, double2* const* x, double tol,
                            const vie_solve_opts* o, vie_solve_info* infos, vie_precond_fn precond,
                            void* const* precond_ctx, cudaStream_t s, int jm = 0);

}  // namespace vie
