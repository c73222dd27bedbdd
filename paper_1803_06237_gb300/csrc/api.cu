// C ABI entry points: plan lifecycle, contrast, operator application.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <chrono>

#include <vector>

#include "vie_internal.cuh"

namespace vie {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

int smooth_size_at_least(int n) {
  if (n < 1) n = 1;
  for (int m = n;; ++m) {
    int r = m;
    while (r % 2 == 0) r /= 2;
    while (r % 3 == 0) r /= 3;
    while (r % 5 == 0) r /= 5;
    if (r == 1) return m;
  }
}

bool factor_length(int len, AxisPlan* out) {
  out->len = len;
  out->nstages = 0;
  int r = len;
  auto push = [&](int f) {
    if (out->nstages >= kMaxStages) return false;
    out->radix[out->nstages++] = f;
    r /= f;
    return true;
  };
  while (r % 4 == 0) if (!push(4)) return false;
  while (r % 2 == 0) if (!push(2)) return false;
  while (r % 3 == 0) if (!push(3)) return false;
  while (r % 5 == 0) if (!push(5)) return false;
  return r == 1;
}

// Radices for lengths with any prime factors: 4, 2, 3, 5 first, then every
// larger prime factor in increasing order (a generic Stockham stage sums
// those directly).  Used by the FFTs along x of the block-circulant
// preconditioner, whose length is the grid's nx.
bool factor_length_any(int len, AxisPlan* out) {
  if (len < 1) return false;
  out->len = len;
  out->nstages = 0;
  int r = len;
  for (int f : {4, 2, 3, 5}) {
    while (r % f == 0) {
      if (out->nstages >= kMaxStages) return false;
      out->radix[out->nstages++] = f;
      r /= f;
    }
  }
  for (int f = 7; r > 1; f += 2) {
    if ((long long)f * f > r) f = r;       // what is left is prime
    while (r % f == 0) {
      if (out->nstages >= kMaxStages) return false;
      out->radix[out->nstages++] = f;
      r /= f;
    }
  }
  return true;
}

// Twiddles exp(-2 pi i k / len) in FP64 on the host (libm cos/sin), the
// argument reduced to the first octant through the symmetries of the circle.
static void twiddle_host(int len, std::vector<double>& re, std::vector<double>& im) {
  re.resize(len);
  im.resize(len);
  for (int k = 0; k < len; ++k) {
    // angle = 2 pi k / len; use k' = 8k mod 8len to find the octant
    const long long num = 8LL * k;          // angle / (pi/4) = num / len
    const int oct = (int)(num / len);       // 0..7
    const long long rem = num - (long long)oct * len;   // in [0, len)
    // residual angle in [0, pi/4): theta = (pi/4) * rem / len
    const double th = (M_PI / 4.0) * (double)rem / (double)len;
    const double c = cos(th), s = sin(th);
    const double h = M_SQRT1_2;
    double cr, sr;   // cos and sin of the full angle
    switch (oct) {
      case 0: cr = c; sr = s; break;
      case 1: cr = h * (c - s); sr = h * (c + s); break;
      case 2: cr = -s; sr = c; break;
      case 3: cr = -h * (c + s); sr = h * (c - s); break;
      case 4: cr = -c; sr = -s; break;
      case 5: cr = -h * (c - s); sr = -h * (c + s); break;
      case 6: cr = s; sr = -c; break;
      default: cr = h * (c + s); sr = -h * (c - s); break;
    }
    re[k] = cr;
    im[k] = -sr;
  }
}

static vie_status make_axis(AxisPlan* ax, int len, size_t* bytes) {
  if (!factor_length(len, ax)) {
    set_error("circulant length %d has a prime factor other than 2, 3, 5", len);
    return VIE_ERR_INVALID;
  }
  std::vector<double> re, im;
  twiddle_host(len, re, im);
  std::vector<double2> t64(len);
  std::vector<float2> t32(len);
  for (int k = 0; k < len; ++k) {
    t64[k] = make_double2(re[k], im[k]);
    t32[k] = make_float2((float)re[k], (float)im[k]);
  }
  VIE_CUDA_TRY(cudaMalloc((void**)&ax->tw64, len * sizeof(double2)));
  VIE_CUDA_TRY(cudaMalloc((void**)&ax->tw32, len * sizeof(float2)));
  VIE_CUDA_TRY(cudaMemcpy(ax->tw64, t64.data(), len * sizeof(double2), cudaMemcpyHostToDevice));
  VIE_CUDA_TRY(cudaMemcpy(ax->tw32, t32.data(), len * sizeof(float2), cudaMemcpyHostToDevice));
  *bytes += len * (sizeof(double2) + sizeof(float2));
  return VIE_OK;
}

// ---------------------------------------------------------------------------
// contrast (step a1): chi = eps/eps_bg - 1 with absorber loss, M = chi/(1+chi)
// ---------------------------------------------------------------------------
constexpr int kMaxAbsorbers = 8;
struct AbsorberSet {
  int n;
  vie_absorber a[kMaxAbsorbers];
};

__global__ void contrast_kernel(double2* __restrict__ chi_io, double2* __restrict__ M64, float2* __restrict__ M32,
                                int nx, size_t N, int from_eps, double eps_bg, AbsorberSet abs_,
                                int* __restrict__ bad) {
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
    double2 e = chi_io[v];
    double cr, ci;
    if (from_eps) {
      const bool core = (e.x != eps_bg) || (e.y != 0.0);
      if (core) {
        const double xc = (double)(v % nx) + 0.5;
        for (int k = 0; k < abs_.n; ++k) {
          const vie_absorber& a = abs_.a[k];
          const double u = a.direction > 0 ? (xc - a.x0) / a.length : (a.x0 - xc) / a.length;
          if (u >= 0.0 && u <= 1.0) {
            double pw = 1.0;
            for (int d = 0; d < a.degree; ++d) pw *= u;
            e.y -= a.eps2_max * pw;
          }
        }
      }
      cr = e.x / eps_bg - 1.0;
      ci = e.y / eps_bg;
    } else {
      cr = e.x;
      ci = e.y;
    }
    // M = chi / (1 + chi)
    const double dr = 1.0 + cr, di = ci;
    const double den = dr * dr + di * di;
    double mr = (cr * dr + ci * di) / den;
    double mi = (ci * dr - cr * di) / den;
    if (!(isfinite(mr) && isfinite(mi)) || den == 0.0) {
      atomicExch(bad, 1);
      mr = 0.0;
      mi = 0.0;
    }
    chi_io[v] = make_double2(cr, ci);
    M64[v] = make_double2(mr, mi);
    M32[v] = make_float2((float)mr, (float)mi);
  }
}

static vie_status set_contrast_common(vie_plan* p, const double* host, const vie_absorber* abs_, int n_abs,
                                      int from_eps) {
  if (!p || !host) { set_error("null argument"); return VIE_ERR_INVALID; }
  if (n_abs < 0 || n_abs > kMaxAbsorbers || (n_abs > 0 && !abs_)) {
    set_error("n_abs must be in [0, %d] with a non-null array", kMaxAbsorbers);
    return VIE_ERR_INVALID;
  }
  AbsorberSet set;
  memset(&set, 0, sizeof(set));
  set.n = n_abs;
  for (int k = 0; k < n_abs; ++k) {
    if (!(abs_[k].length > 0.0) || abs_[k].degree < 0 || (abs_[k].direction != 1 && abs_[k].direction != -1)) {
      set_error("absorber %d: need length > 0, degree >= 0, direction +1 or -1", k);
      return VIE_ERR_INVALID;
    }
    set.a[k] = abs_[k];
  }
  VIE_CUDA_TRY(cudaSetDevice(p->device));
  const size_t N = (size_t)p->n[0] * p->n[1] * p->n[2];
  int* bad = nullptr;
  VIE_CUDA_TRY(cudaMalloc((void**)&bad, sizeof(int)));
  vie_status st = VIE_OK;
  int hbad = 0;
  cudaError_t e = cudaMemset(bad, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(p->chi64, host, N * sizeof(double2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const unsigned blocks = (unsigned)((N + 255) / 256 < 152 * 16 ? (N + 255) / 256 : 152 * 16);
    contrast_kernel<<<blocks, 256>>>(p->chi64, p->M64, p->M32, p->n[0], N, from_eps, p->eps_bg, set, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(bad);
  ++p->contrast_gen;          // preconditioners built from the old contrast are stale
  if (e != cudaSuccess) {
    set_error("set contrast: %s", cudaGetErrorString(e));
    st = VIE_ERR_CUDA;
  } else if (hbad) {
    set_error("contrast is not finite (eps_r = 0 or non-finite input)");
    st = VIE_ERR_NONFINITE;
  }
  return st;
}

// JM-VIE contrast (Sec. 3): mu_r per voxel from the caller, or matched to
// the permittivity's loss (Sec. 4.2, mu'' = eps''/eps' with eps' - j eps'' =
// eps_bg (1 + chi)); M_mu = (mu_r - 1)/mu_r.  The 6N contrast holds M_eps for
// the three electric and M_mu for the three magnetic components.
__global__ void jm_contrast_kernel(const double2* __restrict__ mu_in, const double2* __restrict__ chi,
                                   const double2* __restrict__ Me, double2* __restrict__ chimu,
                                   double2* __restrict__ M64, float2* __restrict__ M32, size_t N, int* bad) {
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
    double2 mu;
    if (mu_in) {
      mu = mu_in[v];
    } else {
      const double2 c = chi[v];
      mu = make_double2(1.0, c.y < 0.0 ? c.y / (1.0 + c.x) : 0.0);   // 1 - j (-Im chi)/(1 + Re chi)
    }
    const double den = mu.x * mu.x + mu.y * mu.y;
    // (mu - 1)/mu = 1 - conj(mu)/|mu|^2
    double mr = 1.0 - mu.x / den, mi = mu.y / den;
    if (!(isfinite(mr) && isfinite(mi)) || den == 0.0) {
      atomicExch(bad, 1);
      mr = 0.0;
      mi = 0.0;
    }
    chimu[v] = make_double2(mu.x - 1.0, mu.y);
    const double2 me = Me[v];
    for (int c = 0; c < 3; ++c) {
      M64[c * N + v] = me;
      M32[c * N + v] = make_float2((float)me.x, (float)me.y);
      M64[(3 + c) * N + v] = make_double2(mr, mi);
      M32[(3 + c) * N + v] = make_float2((float)mr, (float)mi);
    }
  }
}

static void free_plan(vie_plan* p) {
  if (!p) return;
  free_krylov(p);
  free_precond(p);
  bool last = true;
  if (p->shared_refs) {
    last = (--*p->shared_refs == 0);
    if (last) delete p->shared_refs;
  }
  if (last) {
    for (int a = 0; a < 3; ++a) {
      cudaFree(p->ax[a].tw32);
      cudaFree(p->ax[a].tw64);
    }
    cudaFree(p->toeplitz);
    cudaFree(p->ghat64);
    cudaFree(p->ghat32);
  }
  cudaFree(p->M64);
  cudaFree(p->M32);
  cudaFree(p->chi64);
  cudaFree(p->work);
  cudaFree(p->host_stage);
  cudaFree(p->curl);
  cudaFree(p->chat64);
  cudaFree(p->chat32);
  cudaFree(p->Mjm64);
  cudaFree(p->Mjm32);
  cudaFree(p->chimu64);
  cudaFree(p->jm_work);
  delete p;
}

}  // namespace vie

using namespace vie;

// VIE_PLAN_AUTOTUNE: every combination of the three smallest 5-smooth
// sizes >= 2n - 1 per axis and of the compiled x-pass shapes (four-step or
// three-factor, lines per block) for the forward and for the inverse x pass
// is timed (3 warm-up applications, then the best of two bursts of 10
// complex64 operator applications, CUDA events) on a zero spectrum and
// contrast (the time does not depend on the values); the fastest is kept if
// it beats the default configuration by more than 2 %.  Under a profiler
// that serialises kernels the timings, and so the choice, are not those of a
// plain run.  Candidates the passes reject (shared-memory limits) are
// skipped.
static vie_status autotune(vie_plan* p, cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  int cand[3][3];
  for (int a = 0; a < 3; ++a) {
    int m = 2 * p->n[a] - 1;
    for (int c = 0; c < 3; ++c) {
      m = smooth_size_at_least(m);
      cand[a][c] = m;
      ++m;
    }
  }
  const size_t N = (size_t)p->n[0] * p->n[1] * p->n[2];
  const size_t NL = (size_t)3 * p->n[1] * p->n[2];
  const size_t G = (size_t)(cand[0][2] / 2 + 1) * 6 * (cand[1][2] / 2 + 1) * (cand[2][2] / 2 + 1);
  float2 *ghat = nullptr, *M = nullptr, *x = nullptr, *y = nullptr, *work = nullptr;
  AxisPlan ax[3][3];
  size_t scratch = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  vie_status st = VIE_OK;
  auto cleanup = [&]() {
    cudaFree(ghat); cudaFree(M); cudaFree(x); cudaFree(y); cudaFree(work);
    for (auto& row : ax)
      for (auto& a : row) { cudaFree(a.tw32); cudaFree(a.tw64); a = AxisPlan(); }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    p->ghat32 = nullptr;
    p->M32 = nullptr;
    for (int a = 0; a < 3; ++a) p->ax[a] = AxisPlan();
  };
  cudaError_t e = cudaMalloc((void**)&ghat, G * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&M, N * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&x, 3 * N * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&y, 3 * N * sizeof(float2));
  size_t split = 0;
  for (int cx = 0; cx < 3; ++cx)
    for (int cy = 0; cy < 3; ++cy)
      for (int cz = 0; cz < 3; ++cz) {
        const size_t e2 = pass_b_split_elems(p->n[1], p->n[2], cand[0][cx], cand[1][cy], cand[2][cz]);
        if (e2 > split) split = e2;
      }
  const size_t work_bytes = (NL * cand[0][2] + split) * sizeof(float2);
  if (e == cudaSuccess) e = cudaMalloc((void**)&work, work_bytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(ghat, 0, G * sizeof(float2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(M, 0, N * sizeof(float2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, 3 * N * sizeof(float2), s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    set_error("autotune buffers: %s", cudaGetErrorString(e));
    cleanup();
    return e == cudaErrorMemoryAllocation ? VIE_ERR_OOM : VIE_ERR_CUDA;
  }
  for (int a = 0; a < 3 && st == VIE_OK; ++a)
    for (int c = 0; c < 3 && st == VIE_OK; ++c) st = make_axis(&ax[a][c], cand[a][c], &scratch);
  if (st != VIE_OK) { cleanup(); return st; }
  p->ghat32 = ghat;
  p->M32 = M;
  float best = 1e30f;
  int bm[3] = {p->m[0], p->m[1], p->m[2]}, blpb = 0, blpbi = 0, count = 0;
  // time the plan's present configuration: > 0 the best burst in ms, 0 when
  // a pass rejected it, < 0 on a CUDA error (the message is set)
  auto measure = [&]() -> float {
    vie_status ms = VIE_OK;
    for (int r = 0; r < 3 && ms == VIE_OK; ++r) ms = matvec_impl(p, x, y, VIE_C64, MODE_OPERATOR, work, work_bytes, s);
    float t = 1e30f;
    for (int rep = 0; rep < 2 && ms == VIE_OK; ++rep) {   // best of two bursts
      cudaEventRecord(e0, s);
      for (int r = 0; r < 10 && ms == VIE_OK; ++r) ms = matvec_impl(p, x, y, VIE_C64, MODE_OPERATOR, work, work_bytes, s);
      cudaEventRecord(e1, s);
      const cudaError_t se = cudaStreamSynchronize(s);
      if (se != cudaSuccess) {
        set_error("autotune: %s", cudaGetErrorString(se));
        return -1.f;
      }
      float tr = 0.f;
      cudaEventElapsedTime(&tr, e0, e1);
      if (tr < t) t = tr;
    }
    if (ms != VIE_OK) { clear_error(); return 0.f; }
    ++count;
    return t;
  };
  auto set_config = [&](int cx, int cy, int cz) {
    p->m[0] = cand[0][cx];
    p->m[1] = cand[1][cy];
    p->m[2] = cand[2][cz];
    for (int a = 0; a < 3; ++a) p->kf[a] = p->m[a] / 2 + 1;
    p->ax[0] = ax[0][cx];
    p->ax[1] = ax[1][cy];
    p->ax[2] = ax[2][cz];
  };
  // the default configuration first (smallest sizes, heuristic x passes):
  // a candidate replaces it only when more than 2 % faster, so that timing
  // noise between near-equal shapes does not change the plan from run to run
  set_config(0, 0, 0);
  p->x_lpb = 0;
  p->x_lpb_inv = 0;
  const float t_default = measure();
  if (t_default < 0.f) { cleanup(); return VIE_ERR_CUDA; }
  for (int cx = 0; cx < 3; ++cx)
    for (int cy = 0; cy < 3; ++cy)
      for (int cz = 0; cz < 3; ++cz) {
        set_config(cx, cy, cz);
        int l1 = 0, l2 = 0, a1 = 0, a2 = 0, a3 = 0;
        x4_factors(p->m[0], &l1, &l2);
        x3_factors(p->m[0], &a1, &a2, &a3);
        // x-pass variants: four-step with 2 or 4 lines per block, three-factor
        // with 1 or 2 (negative codes), and 5 of either where five-line blocks
        // fill the SMs once, for the forward and the inverse pass
        std::vector<int> modes;
        const bool five = x_lines_five((long)NL, 1) && p->n[0] == 600;
        if (l1) { modes.push_back(2); modes.push_back(4); if (five) modes.push_back(5); }
        if (a1) { modes.push_back(-1); modes.push_back(-2); if (five) modes.push_back(-5); }
        if (modes.empty()) modes.push_back(0);
        const int nm = (int)modes.size();
        for (int li = 0; li < nm * nm; ++li) {   // (forward, inverse) variants
          p->x_lpb = modes[li % nm];
          p->x_lpb_inv = modes[li / nm];
          const float t = measure();
          if (t < 0.f) { cleanup(); return VIE_ERR_CUDA; }
          if (t > 0.f && t < best) {
            best = t;
            bm[0] = p->m[0]; bm[1] = p->m[1]; bm[2] = p->m[2];
            blpb = p->x_lpb;
            blpbi = p->x_lpb_inv;
          }
        }
      }
  if (t_default > 0.f && !(best < 0.98f * t_default)) {
    for (int a = 0; a < 3; ++a) bm[a] = cand[a][0];
    blpb = 0;
    blpbi = 0;
  }
  cleanup();
  if (count == 0) { set_error("autotune: no candidate configuration ran"); return VIE_ERR_INVALID; }
  for (int a = 0; a < 3; ++a) {
    p->m[a] = bm[a];
    p->kf[a] = bm[a] / 2 + 1;
  }
  p->x_lpb = blpb;
  p->x_lpb_inv = blpbi;
  p->tune_candidates = count;
  p->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return VIE_OK;
}

extern "C" {

const char* vie_last_error(void) { return g_err; }

vie_status vie_plan_create(vie_plan** out, const int n[3], double h, double k0, double eps_bg, int flags) {
  clear_error();
  if (!out || !n) { set_error("null argument"); return VIE_ERR_INVALID; }
  *out = nullptr;
  if (n[0] < 1 || n[1] < 1 || n[2] < 1) { set_error("grid sizes must be >= 1"); return VIE_ERR_INVALID; }
  if (!(h > 0.0) || !(k0 >= 0.0) || !(eps_bg > 0.0) || !isfinite(h) || !isfinite(k0) || !isfinite(eps_bg)) {
    set_error("need h > 0, k0 >= 0, eps_bg > 0 (finite)");
    return VIE_ERR_INVALID;
  }
  if ((double)n[0] * n[1] * n[2] > 2.0e9) { set_error("grid too large"); return VIE_ERR_INVALID; }
  vie_plan* p = new vie_plan();
  VIE_CUDA_TRY(cudaGetDevice(&p->device));
  for (int a = 0; a < 3; ++a) {
    p->n[a] = n[a];
    p->m[a] = (flags & VIE_PLAN_CIRC_2N) ? 2 * n[a] : smooth_size_at_least(2 * n[a] - 1);
    p->kf[a] = p->m[a] / 2 + 1;
  }
  p->h = h;
  p->k0 = k0;
  p->eps_bg = eps_bg;
  p->kappa = k0 * sqrt(eps_bg) * h;
  size_t bytes = 0;
  vie_status st = VIE_OK;
  if ((flags & VIE_PLAN_AUTOTUNE) && !(flags & VIE_PLAN_CIRC_2N)) {
    cudaStream_t ts;
    if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("cudaStreamCreate failed");
      free_plan(p);
      return VIE_ERR_CUDA;
    }
    st = autotune(p, ts);
    cudaStreamDestroy(ts);
    if (st != VIE_OK) { free_plan(p); return st; }
  }
  for (int a = 0; a < 3 && st == VIE_OK; ++a) st = make_axis(&p->ax[a], p->m[a], &bytes);
  if (st != VIE_OK) { free_plan(p); return st; }
  const size_t N = (size_t)n[0] * n[1] * n[2];
  const size_t G = (size_t)p->kf[0] * 6 * p->kf[1] * p->kf[2];
  const size_t NL = (size_t)3 * n[1] * n[2];
  p->work_bytes = (NL * p->m[0] + pass_b_split_elems(n[1], n[2], p->m[0], p->m[1], p->m[2])) * sizeof(double2);
  struct { void** ptr; size_t sz; } allocs[] = {
      {(void**)&p->toeplitz, 6 * N * sizeof(double2)}, {(void**)&p->ghat64, G * sizeof(double2)},
      {(void**)&p->ghat32, G * sizeof(float2)},        {(void**)&p->M64, N * sizeof(double2)},
      {(void**)&p->M32, N * sizeof(float2)},           {(void**)&p->chi64, N * sizeof(double2)},
      {(void**)&p->work, p->work_bytes}};
  for (auto& a : allocs) {
    cudaError_t e = cudaMalloc(a.ptr, a.sz);
    if (e != cudaSuccess) {
      set_error("cudaMalloc(%zu) failed: %s", a.sz, cudaGetErrorString(e));
      free_plan(p);
      return e == cudaErrorMemoryAllocation ? VIE_ERR_OOM : VIE_ERR_CUDA;
    }
    bytes += a.sz;
  }
  p->device_bytes = bytes;
  cudaStream_t s;
  cudaEvent_t e0, e1;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("cudaStreamCreate failed");
    free_plan(p);
    return VIE_ERR_CUDA;
  }
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  cudaMemsetAsync(p->M64, 0, N * sizeof(double2), s);
  cudaMemsetAsync(p->M32, 0, N * sizeof(float2), s);
  cudaMemsetAsync(p->chi64, 0, N * sizeof(double2), s);
  st = compute_toeplitz(p, s);
  if (st == VIE_OK) st = compute_spectrum(p, s);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (st == VIE_OK && e != cudaSuccess) {
    set_error("plan setup failed: %s", cudaGetErrorString(e));
    st = VIE_ERR_CUDA;
  }
  float ms = 0.f;
  if (st == VIE_OK) cudaEventElapsedTime(&ms, e0, e1);
  p->setup_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (st == VIE_OK) st = static_scratch_prepare();
  if (st != VIE_OK) { free_plan(p); return st; }
  *out = p;
  return VIE_OK;
}

vie_status vie_plan_clone(const vie_plan* base, vie_plan** out) {
  clear_error();
  if (!base || !out) { set_error("null argument"); return VIE_ERR_INVALID; }
  *out = nullptr;
  VIE_CUDA_TRY(cudaSetDevice(base->device));
  vie_plan* p = new vie_plan();
  for (int a = 0; a < 3; ++a) {
    p->n[a] = base->n[a];
    p->m[a] = base->m[a];
    p->x_lpb = base->x_lpb;
    p->x_lpb_inv = base->x_lpb_inv;
    p->kf[a] = base->kf[a];
    p->ax[a] = base->ax[a];
  }
  p->h = base->h;
  p->k0 = base->k0;
  p->eps_bg = base->eps_bg;
  p->kappa = base->kappa;
  p->device = base->device;
  p->toeplitz = base->toeplitz;
  p->ghat64 = base->ghat64;
  p->ghat32 = base->ghat32;
  p->setup_ms = 0.0;
  vie_plan* b = const_cast<vie_plan*>(base);
  if (!b->shared_refs) b->shared_refs = new int(1);
  p->shared_refs = b->shared_refs;
  ++*p->shared_refs;
  const size_t N = (size_t)p->n[0] * p->n[1] * p->n[2];
  p->work_bytes = base->work_bytes;
  struct { void** ptr; size_t sz; } allocs[] = {
      {(void**)&p->M64, N * sizeof(double2)}, {(void**)&p->M32, N * sizeof(float2)},
      {(void**)&p->chi64, N * sizeof(double2)}, {(void**)&p->work, p->work_bytes}};
  size_t bytes = 0;
  for (auto& a : allocs) {
    cudaError_t e = cudaMalloc(a.ptr, a.sz);
    if (e != cudaSuccess) {
      set_error("cudaMalloc(%zu) failed: %s", a.sz, cudaGetErrorString(e));
      free_plan(p);
      return e == cudaErrorMemoryAllocation ? VIE_ERR_OOM : VIE_ERR_CUDA;
    }
    bytes += a.sz;
  }
  p->device_bytes = bytes;
  cudaError_t e = cudaMemset(p->M64, 0, N * sizeof(double2));
  if (e == cudaSuccess) e = cudaMemset(p->M32, 0, N * sizeof(float2));
  if (e == cudaSuccess) e = cudaMemset(p->chi64, 0, N * sizeof(double2));
  if (e != cudaSuccess) {
    set_error("cudaMemset failed: %s", cudaGetErrorString(e));
    free_plan(p);
    return VIE_ERR_CUDA;
  }
  vie_status st = static_scratch_prepare();
  if (st != VIE_OK) { free_plan(p); return st; }
  *out = p;
  return VIE_OK;
}

vie_status vie_matvec_batch(vie_plan* const* plans, int count, const void* const* x, void* const* y, int dtype,
                            void* stream) {
  clear_error();
  if (!plans || !x || !y || count < 1) { set_error("null argument or count < 1"); return VIE_ERR_INVALID; }
  if (dtype != VIE_C64 && dtype != VIE_C128) { set_error("dtype must be VIE_C64 or VIE_C128"); return VIE_ERR_INVALID; }
  for (int i = 0; i < count; ++i) {
    if (!plans[i] || !x[i] || !y[i]) { set_error("null plan or vector %d", i); return VIE_ERR_INVALID; }
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) { set_error("plan %d appears twice (its workspace would be shared)", i); return VIE_ERR_INVALID; }
  }
  // group plans of one shape, keeping the caller's order inside a group
  std::vector<int> done(count, 0);
  for (int i = 0; i < count; ++i) {
    if (done[i]) continue;
    std::vector<vie_plan*> gp;
    std::vector<const void*> gx;
    std::vector<void*> gy;
    for (int j = i; j < count; ++j) {
      if (done[j]) continue;
      const vie_plan* a = plans[i];
      const vie_plan* b = plans[j];
      if (a->n[0] == b->n[0] && a->n[1] == b->n[1] && a->n[2] == b->n[2] && a->m[0] == b->m[0] &&
          a->m[1] == b->m[1] && a->m[2] == b->m[2] && a->device == b->device) {
        gp.push_back(plans[j]);
        gx.push_back(x[j]);
        gy.push_back(y[j]);
        done[j] = 1;
      }
    }
    vie_status st = matvec_group(gp.data(), (int)gp.size(), gx.data(), gy.data(), dtype, MODE_OPERATOR,
                                 (cudaStream_t)stream);
    if (st != VIE_OK) return st;
  }
  return VIE_OK;
}

vie_status vie_plan_destroy(vie_plan* plan) {
  clear_error();
  if (!plan) return VIE_OK;
  cudaSetDevice(plan->device);
  free_plan(plan);
  return VIE_OK;
}

vie_status vie_plan_get_info(const vie_plan* p, vie_plan_info* info) {
  clear_error();
  if (!p || !info) { set_error("null argument"); return VIE_ERR_INVALID; }
  for (int a = 0; a < 3; ++a) { info->n[a] = p->n[a]; info->m[a] = p->m[a]; }
  info->h = p->h;
  info->k0 = p->k0;
  info->eps_bg = p->eps_bg;
  info->kappa = p->kappa;
  info->device_bytes = p->device_bytes;
  info->setup_ms = p->setup_ms;
  info->tune_ms = p->tune_ms;
  info->tune_candidates = p->tune_candidates;
  info->x_lines_per_block = p->x_lpb;
  info->x_lines_per_block_inverse = p->x_lpb_inv;
  return VIE_OK;
}

vie_status vie_set_permittivity(vie_plan* p, const double* eps_host, const vie_absorber* absorbers, int n_abs) {
  clear_error();
  return set_contrast_common(p, eps_host, absorbers, n_abs, 1);
}

vie_status vie_set_contrast(vie_plan* p, const double* chi_host) {
  clear_error();
  return set_contrast_common(p, chi_host, nullptr, 0, 0);
}

static vie_status check_vec_args(vie_plan* p, const void* x, void* y, int dtype) {
  if (!p || !x || !y) { set_error("null argument"); return VIE_ERR_INVALID; }
  if (dtype != VIE_C64 && dtype != VIE_C128) { set_error("dtype must be VIE_C64 or VIE_C128"); return VIE_ERR_INVALID; }
  const size_t bytes = (size_t)3 * p->n[0] * p->n[1] * p->n[2] * (dtype == VIE_C64 ? 8 : 16);
  const char* a = (const char*)x;
  const char* b = (const char*)y;
  if (a < b + bytes && b < a + bytes) { set_error("x and y overlap"); return VIE_ERR_INVALID; }
  return VIE_OK;
}

vie_status vie_matvec(vie_plan* p, const void* x, void* y, int dtype, void* stream) {
  clear_error();
  vie_status st = check_vec_args(p, x, y, dtype);
  if (st != VIE_OK) return st;
  return matvec_impl(p, x, y, dtype, MODE_OPERATOR, p->work, p->work_bytes, (cudaStream_t)stream);
}

vie_status vie_rhs_from_source(vie_plan* p, const void* src, void* b, int dtype, void* stream) {
  clear_error();
  vie_status st = check_vec_args(p, src, b, dtype);
  if (st != VIE_OK) return st;
  return matvec_impl(p, src, b, dtype, MODE_RHS, p->work, p->work_bytes, (cudaStream_t)stream);
}

vie_status vie_get_toeplitz(const vie_plan* p, double* out) {
  clear_error();
  if (!p || !out) { set_error("null argument"); return VIE_ERR_INVALID; }
  const size_t N = (size_t)p->n[0] * p->n[1] * p->n[2];
  VIE_CUDA_TRY(cudaSetDevice(p->device));
  VIE_CUDA_TRY(cudaMemcpy(out, p->toeplitz, 6 * N * sizeof(double2), cudaMemcpyDeviceToHost));
  return VIE_OK;
}

vie_status vie_set_permeability(vie_plan* p, const double* mu_host) {
  clear_error();
  if (!p) { set_error("null plan"); return VIE_ERR_INVALID; }
  VIE_CUDA_TRY(cudaSetDevice(p->device));
  const size_t N = (size_t)p->n[0] * p->n[1] * p->n[2];
  if (!p->curl) {
    // first call: the curl entries, their spectra, the 6N contrast and the workspace
    const size_t C = (size_t)p->kf[0] * 3 * p->kf[1] * p->kf[2];
    const size_t W = (size_t)6 * p->n[1] * p->n[2] * p->m[0];
    struct { void** ptr; size_t sz; } allocs[] = {
        {(void**)&p->curl, 3 * N * sizeof(double2)}, {(void**)&p->chat64, C * sizeof(double2)},
        {(void**)&p->chat32, C * sizeof(float2)},    {(void**)&p->Mjm64, 6 * N * sizeof(double2)},
        {(void**)&p->Mjm32, 6 * N * sizeof(float2)}, {(void**)&p->chimu64, N * sizeof(double2)},
        {(void**)&p->jm_work, W * sizeof(double2)}};
    for (auto& a : allocs) {
      cudaError_t e = cudaMalloc(a.ptr, a.sz);
      if (e != cudaSuccess) {
        set_error("cudaMalloc(%zu) for the JM-VIE: %s", a.sz, cudaGetErrorString(e));
        for (auto& b : allocs) { cudaFree(*b.ptr); *b.ptr = nullptr; }
        return e == cudaErrorMemoryAllocation ? VIE_ERR_OOM : VIE_ERR_CUDA;
      }
      p->device_bytes += a.sz;
    }
    vie_status st = compute_curl(p, 0);
    if (st == VIE_OK) {
      cudaError_t e = cudaDeviceSynchronize();
      if (e != cudaSuccess) { set_error("curl spectrum: %s", cudaGetErrorString(e)); st = VIE_ERR_CUDA; }
    }
    if (st != VIE_OK) {
      cudaFree(p->curl);
      p->curl = nullptr;
      return st;
    }
  }
  double2* mu_dev = nullptr;
  int* bad = nullptr;
  VIE_CUDA_TRY(cudaMalloc((void**)&bad, sizeof(int)));
  cudaError_t e = cudaMemset(bad, 0, sizeof(int));
  if (e == cudaSuccess && mu_host) {
    e = cudaMalloc((void**)&mu_dev, N * sizeof(double2));
    if (e == cudaSuccess) e = cudaMemcpy(mu_dev, mu_host, N * sizeof(double2), cudaMemcpyHostToDevice);
  }
  int hbad = 0;
  if (e == cudaSuccess) {
    const unsigned blocks = (unsigned)((N + 255) / 256 < 152 * 16 ? (N + 255) / 256 : 152 * 16);
    jm_contrast_kernel<<<blocks, 256>>>(mu_dev, p->chi64, p->M64, p->chimu64, p->Mjm64, p->Mjm32, N, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(bad);
  cudaFree(mu_dev);
  if (e != cudaSuccess) {
    set_error("set permeability: %s", cudaGetErrorString(e));
    return VIE_ERR_CUDA;
  }
  if (hbad) {
    set_error("permeability is not finite or zero");
    return VIE_ERR_NONFINITE;
  }
  p->jm_gen = p->contrast_gen;
  return VIE_OK;
}

static vie_status check_jm_args(vie_plan* p, const void* x, void* y, int dtype) {
  if (!p || !x || !y) { set_error("null argument"); return VIE_ERR_INVALID; }
  if (dtype != VIE_C64 && dtype != VIE_C128) { set_error("dtype must be VIE_C64 or VIE_C128"); return VIE_ERR_INVALID; }
  if (!p->curl) { set_error("call vie_set_permeability before the JM-VIE operator"); return VIE_ERR_INVALID; }
  if (p->jm_gen != p->contrast_gen) {
    set_error("the permittivity changed after vie_set_permeability: call it again");
    return VIE_ERR_INVALID;
  }
  const size_t bytes = (size_t)6 * p->n[0] * p->n[1] * p->n[2] * (dtype == VIE_C64 ? 8 : 16);
  const char* a = (const char*)x;
  const char* b = (const char*)y;
  if (a < b + bytes && b < a + bytes) { set_error("x and y overlap"); return VIE_ERR_INVALID; }
  return VIE_OK;
}

vie_status vie_jm_matvec(vie_plan* p, const void* x, void* y, int dtype, void* stream) {
  clear_error();
  vie_status st = check_jm_args(p, x, y, dtype);
  if (st != VIE_OK) return st;
  return jm_matvec_impl(p, x, y, dtype, MODE_OPERATOR, (cudaStream_t)stream);
}

vie_status vie_jm_rhs_from_source(vie_plan* p, const void* src, void* b, int dtype, void* stream) {
  clear_error();
  vie_status st = check_jm_args(p, src, b, dtype);
  if (st != VIE_OK) return st;
  return jm_matvec_impl(p, src, b, dtype, MODE_RHS, (cudaStream_t)stream);
}

vie_status vie_eps2_from_round_trip(double r_rt, int degree, double length, double k0, double eps_r, double D,
                                    double eta, double* eps2_max) {
  clear_error();
  if (!eps2_max || !(r_rt > 0.0 && r_rt < 1.0) || degree < 0 || !(length > 0.0) || !(k0 > 0.0) ||
      !(eps_r > 0.0) || !(D > 0.0) || !(eta > 0.0)) {
    set_error("need 0 < r_rt < 1, degree >= 0 and positive length, k0, eps_r, D, eta");
    return VIE_ERR_INVALID;
  }
  *eps2_max = -(degree + 1) * log(r_rt) * sqrt(eps_r) / (D * length * eta * k0);
  return VIE_OK;
}

}  // extern "C"
