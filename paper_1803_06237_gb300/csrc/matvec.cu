// The J-VIE operator application y = w - M (N w) (Sec. 5.4 of arXiv:1803.06237:
// the block-Toeplitz N, six unique tensor components, applied with FFTs; the
// diagonal multiplier M_eps of Sec. 3 carries material and absorber).
//
// Three passes over a workspace X[kx][line] (line = (c nz + z) ny + y, the
// 3 ny nz non-zero x-lines of the zero-padded currents):
//   A  per group of x-lines: load nx values, zero-pad to Mx, forward FFT along
//      x, write transposed so that one kx holds all lines contiguously.
//   B  per kx: forward FFT along z (ny non-zero rows) and y (all Mz columns),
//      u_p = sum_q G_pq w_q with the folded spectrum (parity signs restore the
//      other octants), inverse FFT along y (keep y < ny) and z (keep z < nz),
//      written back in place.
//   C  per group of x-lines: inverse FFT along x, crop to nx, and
//      y = w - M u (operator) or y = M (u - w) (right-hand side of a source).
// Planes too large for one CTA's shared memory (My Mz beyond a few thousand,
// e.g. 1200 x 24) split pass B in three launches through a y-pass buffer in
// the plan's workspace (run_split_b: y lines, z stage, inverse y); without
// that buffer (the static workspace) or a z-stage kernel for Mz, pass B runs
// on a cluster of CTAs per kx sharing the plane through distributed shared
// memory (pass_b_cluster_kernel).
// The spectrum is pre-scaled by 1/(Mx My Mz), so no separate normalisation.
#include <cooperative_groups.h>
#include <cuda_pipeline.h>
#include <stdio.h>
#include <string.h>

#include "fft.cuh"
#include "regfft.cuh"
#include "vie_internal.cuh"

namespace vie {

template <typename V> __device__ __forceinline__ V zero_c();
template <> __device__ __forceinline__ float2 zero_c<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 zero_c<double2>() { return make_double2(0.0, 0.0); }

// Per-problem pointers of one launch: blockIdx.y selects the problem.  All
// problems of a launch share the grid and circulant sizes (and twiddles).
constexpr int kMaxBatch = 16;
template <typename V>
struct PassPtrs {
  const V* x[kMaxBatch];
  V* y[kMaxBatch];
  V* work[kMaxBatch];
  const V* ghat[kMaxBatch];
  const V* M[kMaxBatch];
  V* work2[kMaxBatch];        // y-pass buffer of the split pass B (or null)
  const int* live[kMaxBatch]; // per problem: null, or a device flag; 0 skips the problem (its blocks return)
};

// A problem whose live flag is 0 is skipped by every block of every pass
// (blockIdx.y is the problem in all grouped launches).
template <typename V>
__device__ __forceinline__ bool skip_problem(const PassPtrs<V>& pp) {
  const int* f = pp.live[blockIdx.y];
  return f != nullptr && *(const volatile int*)f == 0;
}

// ---------------------------------------------------------------------------
// pass A
// ---------------------------------------------------------------------------
template <typename V>
__global__ void __launch_bounds__(256) pass_a_kernel(const __grid_constant__ PassPtrs<V> pp, int nx, int NL,
                                                     Radices rx, const V* __restrict__ twg, int lines_per_block,
                                                     int gsz) {
  if (skip_problem(pp)) return;
  pdl_wait();
  const V* __restrict__ x = pp.x[blockIdx.y];
  V* __restrict__ work = pp.work[blockIdx.y];
  extern __shared__ unsigned char smem_raw[];
  const int Mx = rx.len;
  const int pitch = Mx + 1;
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* A = tw + Mx;
  V* B = A + (size_t)lines_per_block * pitch;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int l0 = blockIdx.x * lines_per_block;
  const int nl = min(lines_per_block, NL - l0);
  for (int i = tid; i < Mx; i += nth) tw[i] = twg[i];
  for (int e = tid; e < nl * Mx; e += nth) {
    const int l = e / Mx, k = e - l * Mx;
    A[l * pitch + k] = (k < nx) ? x[(size_t)(l0 + l) * nx + k] : zero_c<V>();
  }
  __syncthreads();
  V* res = fft_lines<V, false>(A, B, rx, pitch, nl, tw, tid, nth);
  for (int e = tid; e < nl * Mx; e += nth) {
    const int kx = e / nl, l = e - kx * nl;
    const int line = l0 + l, grp = line / gsz;
    work[((size_t)grp * Mx + kx) * gsz + (line - grp * gsz)] = res[l * pitch + kx];
  }
}

// ---------------------------------------------------------------------------
// pass B
// ---------------------------------------------------------------------------
struct PassBGeom {
  int ny, nz, NL, Mx, My, Mz, Ky, Kz;
};

template <typename V>
__global__ void __launch_bounds__(256) pass_b_kernel(const __grid_constant__ PassPtrs<V> pp, PassBGeom g,
                                                     Radices ry, Radices rz, const V* __restrict__ twyg,
                                                     const V* __restrict__ twzg) {
  if (skip_problem(pp)) return;
  pdl_wait();
  V* __restrict__ work = pp.work[blockIdx.y];
  const V* __restrict__ ghat = pp.ghat[blockIdx.y];
  extern __shared__ unsigned char smem_raw[];
  const int kx = blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int ny = g.ny, nz = g.nz, My = g.My, Mz = g.Mz;
  const int pz = Mz + 1, py = My + 1;
  const int buf = 3 * Mz * py;   // >= 3 * ny * pz since My >= ny
  V* twy = reinterpret_cast<V*>(smem_raw);
  V* twz = twy + My;
  V* U = twz + Mz;
  V* W = U + buf;
  for (int i = tid; i < My; i += nth) twy[i] = twyg[i];
  for (int i = tid; i < Mz; i += nth) twz[i] = twzg[i];
  // load the kx slab: z-rows (c, y) of length Mz, zero-padded
  V* slab = work + (size_t)kx * g.NL;
  for (int e = tid; e < 3 * ny * Mz; e += nth) {
    const int row = e / Mz, z = e - row * Mz;   // row = c*ny + y
    const int c = row / ny, y = row - c * ny;
    U[row * pz + z] = (z < nz) ? slab[(c * nz + z) * ny + y] : zero_c<V>();
  }
  __syncthreads();
  V* zr = fft_lines<V, false>(U, W, rz, pz, 3 * ny, twz, tid, nth);
  V* other = (zr == U) ? W : U;
  // transpose to y-rows (c, kz) of length My, zero-padded
  for (int e = tid; e < 3 * Mz * My; e += nth) {
    const int row = e / My, y = e - row * My;   // row = c*Mz + kz
    const int c = row / Mz, kz = row - c * Mz;
    other[row * py + y] = (y < ny) ? zr[(c * ny + y) * pz + kz] : zero_c<V>();
  }
  __syncthreads();
  V* yr = fft_lines<V, false>(other, zr, ry, py, 3 * Mz, twy, tid, nth);
  // spectral multiply u_p = sum_q G_pq w_q with folded spectrum and parity signs
  {
    const bool fx = kx > g.Mx - kx;
    const int kxf = fx ? g.Mx - kx : kx;
    const V* G = ghat + (size_t)kxf * 6 * g.Kz * g.Ky;
    for (int e = tid; e < Mz * My; e += nth) {
      const int kz = e / My, ky = e - kz * My;
      const bool fy = ky > My - ky, fz = kz > Mz - kz;
      const int kyf = fy ? My - ky : ky, kzf = fz ? Mz - kz : kz;
      const size_t o = (size_t)kzf * g.Ky + kyf;
      const size_t cs = (size_t)g.Kz * g.Ky;
      V gxx = G[o], gyy = G[cs + o], gzz = G[2 * cs + o];
      V gxy = G[3 * cs + o], gxz = G[4 * cs + o], gyz = G[5 * cs + o];
      if (fx ^ fy) gxy = scale(gxy, -1.0f);
      if (fx ^ fz) gxz = scale(gxz, -1.0f);
      if (fy ^ fz) gyz = scale(gyz, -1.0f);
      V* px = yr + (0 * Mz + kz) * py + ky;
      V* pyv = yr + (1 * Mz + kz) * py + ky;
      V* pzv = yr + (2 * Mz + kz) * py + ky;
      const V wx = *px, wy = *pyv, wz = *pzv;
      *px = add(add(mul(gxx, wx), mul(gxy, wy)), mul(gxz, wz));
      *pyv = add(add(mul(gxy, wx), mul(gyy, wy)), mul(gyz, wz));
      *pzv = add(add(mul(gxz, wx), mul(gyz, wy)), mul(gzz, wz));
    }
  }
  __syncthreads();
  V* spare = (yr == U) ? W : U;
  V* yi = fft_lines<V, true>(yr, spare, ry, py, 3 * Mz, twy, tid, nth);
  V* other2 = (yi == U) ? W : U;
  // back to z-rows (c, y < ny) of length Mz
  for (int e = tid; e < 3 * ny * Mz; e += nth) {
    const int row = e / Mz, kz = e - row * Mz;   // row = c*ny + y
    const int c = row / ny, y = row - c * ny;
    other2[row * pz + kz] = yi[(c * Mz + kz) * py + y];
  }
  __syncthreads();
  V* spare2 = (other2 == U) ? W : U;
  V* zi = fft_lines<V, true>(other2, spare2, rz, pz, 3 * ny, twz, tid, nth);
  for (int e = tid; e < g.NL; e += nth) {
    const int y = e % ny, cz = e / ny;
    const int z = cz % nz, c = cz / nz;
    slab[e] = zi[(c * ny + y) * pz + z];
  }
}

// ---------------------------------------------------------------------------
// pass B for y-z planes larger than one CTA's shared memory: a cluster of CS
// CTAs per kx holds the plane in distributed shared memory.
//   1. CTA r loads the y-lines l = c nz + z, l in [r nl, (r + 1) nl), pads
//      them with zeros to My and transforms them along y.
//   2. Cluster barrier.  CTA r takes ky in [r nk, (r + 1) nk), kc at a time:
//      it gathers the 3 nz values of each ky from the owners' shared memory,
//      pads along z, transforms along z, multiplies by the folded 3x3
//      spectrum, transforms back along z and scatters z < nz to the owners.
//   3. Cluster barrier.  Each CTA transforms its own lines back along y and
//      writes y < ny to the workspace slab.
// y goes first because only the 3 nz non-zero lines need it: 3 nz My log My
// + 3 My Mz log Mz operations, against 3 ny Mz log Mz + 3 Mz My log My for z
// first, fewer when ny >> nz (the 600 x 11 cross-section of a ring
// resonator).  Remote accesses walk ky, which is contiguous in the owner's
// rows.  No CTA touches another's shared memory after the last barrier.
// ---------------------------------------------------------------------------
struct ClusterGeom {
  int cs;       // CTAs per cluster (one cluster per kx)
  int nl;       // y-lines per CTA
  int nk;       // ky values per CTA in the z stage
  int kc;       // ky values per chunk of the z stage
  int py, pz;   // shared row pitches (odd)
};

template <typename V>
__global__ void __launch_bounds__(256) pass_b_cluster_kernel(const __grid_constant__ PassPtrs<V> pp, PassBGeom g,
                                                             ClusterGeom q, Radices ry, Radices rz,
                                                             const V* __restrict__ twyg,
                                                             const V* __restrict__ twzg) {
  if (skip_problem(pp)) return;
  namespace cgr = cooperative_groups;
  cgr::cluster_group cluster = cgr::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int kx = blockIdx.x / q.cs;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int ny = g.ny, nz = g.nz, My = g.My, Mz = g.Mz;
  const int nly = 3 * nz;
  const int py = q.py, pz = q.pz, nl = q.nl, kc = q.kc;
  const int l0 = rank * nl;
  const int nown = max(0, min(nly - l0, nl));
  extern __shared__ unsigned char smem_raw[];
  V* twy = reinterpret_cast<V*>(smem_raw);
  V* twz = twy + My;
  V* A = twz + Mz;
  V* B = A + (size_t)nl * py;
  V* Z0 = B + (size_t)nl * py;
  V* Z1 = Z0 + (size_t)3 * kc * pz;
  pdl_launch_dependents();
  for (int i = tid; i < My; i += nth) twy[i] = twyg[i];
  for (int i = tid; i < Mz; i += nth) twz[i] = twzg[i];
  pdl_wait();
  V* __restrict__ slab = pp.work[blockIdx.y] + (size_t)kx * g.NL;
  const V* __restrict__ ghat = pp.ghat[blockIdx.y];
  for (int e = tid; e < nown * My; e += nth) {
    const int row = e / My, y = e - row * My;
    A[row * py + y] = (y < ny) ? slab[(size_t)(l0 + row) * ny + y] : zero_c<V>();
  }
  __syncthreads();
  V* Y = fft_lines<V, false>(A, B, ry, py, nown, twy, tid, nth);   // same buffer in every CTA
  V* spare = (Y == A) ? B : A;
  cluster.sync();

  const bool fx = kx > g.Mx - kx;
  const int kxf = fx ? g.Mx - kx : kx;
  const V* G = ghat + (size_t)kxf * 6 * g.Kz * g.Ky;
  const size_t gcs = (size_t)g.Kz * g.Ky;
  const int kbeg = rank * q.nk, kend = min(My, kbeg + q.nk);
  for (int kb = kbeg; kb < kend; kb += kc) {
    const int kn = min(kc, kend - kb);
    // rows (c, j) of Z0: z < nz from the owners of lines c nz + z, then zeros
    for (int e = tid; e < nly * kn; e += nth) {
      const int l = e / kn, j = e - l * kn;
      const int owner = l / nl;
      const V* src = cluster.map_shared_rank(Y, owner);
      const int c = l / nz, z = l - c * nz;
      Z0[(c * kn + j) * pz + z] = src[(size_t)(l - owner * nl) * py + kb + j];
    }
    for (int e = tid; e < 3 * kn * (Mz - nz); e += nth) {
      const int row = e / (Mz - nz), z = nz + (e - row * (Mz - nz));
      Z0[row * pz + z] = zero_c<V>();
    }
    __syncthreads();
    V* Zf = fft_lines<V, false>(Z0, Z1, rz, pz, 3 * kn, twz, tid, nth);
    for (int e = tid; e < Mz * kn; e += nth) {
      const int kz = e / kn, j = e - kz * kn;
      const int ky = kb + j;
      const bool fy = ky > My - ky, fz = kz > Mz - kz;
      const int kyf = fy ? My - ky : ky, kzf = fz ? Mz - kz : kz;
      const size_t o = (size_t)kzf * g.Ky + kyf;
      V gxx = G[o], gyy = G[gcs + o], gzz = G[2 * gcs + o];
      V gxy = G[3 * gcs + o], gxz = G[4 * gcs + o], gyz = G[5 * gcs + o];
      if (fx ^ fy) gxy = scale(gxy, -1.0f);
      if (fx ^ fz) gxz = scale(gxz, -1.0f);
      if (fy ^ fz) gyz = scale(gyz, -1.0f);
      V* px = Zf + (0 * kn + j) * pz + kz;
      V* pyv = Zf + (1 * kn + j) * pz + kz;
      V* pzv = Zf + (2 * kn + j) * pz + kz;
      const V wx = *px, wy = *pyv, wz = *pzv;
      *px = add(add(mul(gxx, wx), mul(gxy, wy)), mul(gxz, wz));
      *pyv = add(add(mul(gxy, wx), mul(gyy, wy)), mul(gyz, wz));
      *pzv = add(add(mul(gxz, wx), mul(gyz, wy)), mul(gzz, wz));
    }
    __syncthreads();
    V* Zi = fft_lines<V, true>(Zf, (Zf == Z0) ? Z1 : Z0, rz, pz, 3 * kn, twz, tid, nth);
    for (int e = tid; e < nly * kn; e += nth) {
      const int l = e / kn, j = e - l * kn;
      const int owner = l / nl;
      V* dst = cluster.map_shared_rank(Y, owner);
      const int c = l / nz, z = l - c * nz;
      dst[(size_t)(l - owner * nl) * py + kb + j] = Zi[(c * kn + j) * pz + z];
    }
    __syncthreads();
  }
  cluster.sync();
  V* Yi = fft_lines<V, true>(Y, spare, ry, py, nown, twy, tid, nth);
  for (int e = tid; e < nown * ny; e += nth) {
    const int row = e / ny, y = e - row * ny;
    slab[(size_t)(l0 + row) * ny + y] = Yi[row * py + y];
  }
}

// Cluster shape: the smallest cluster whose CTAs fit a shared-memory budget
// with at least 16 ky per z-stage chunk, trying first a budget that leaves
// room for two CTAs per SM, then one CTA per SM, then chunks of any size;
// false when even eight CTAs do not fit.
static bool pass_b_cluster_geom(int nz, int My, int Mz, size_t vbytes, ClusterGeom* out) {
  const long budgets[2] = {(long)(110 * 1024 / vbytes), (long)(220 * 1024 / vbytes)};
  const int py = My | 1, pz = Mz | 1;
  const int nly = 3 * nz;
  for (int want = 16; want >= 1; want -= 15)
    for (int b = 0; b < 2; ++b)
      for (int cs = 2; cs <= 8; ++cs) {
        const int nl = (nly + cs - 1) / cs;
        const int nk = (My + cs - 1) / cs;
        const long base = (long)My + Mz + 2L * nl * py;
        const long kmin = want < nk ? want : nk;
        if (base + 6L * pz * kmin > budgets[b]) continue;
        long kc = (budgets[b] - base) / (6L * pz);
        if (kc > nk) kc = nk;
        if (kc > 64) kc = 64;
        *out = ClusterGeom{cs, nl, nk, (int)kc, py, pz};
        return true;
      }
  return false;
}

static size_t pass_b_cluster_smem(const PassBGeom& g, const ClusterGeom& q, size_t vbytes) {
  return ((size_t)g.My + g.Mz + 2 * (size_t)q.nl * q.py + 6 * (size_t)q.kc * q.pz) * vbytes;
}

template <typename V>
static vie_status launch_pass_b_cluster(const PassPtrs<V>& pp, int count, const PassBGeom& g, Radices ry,
                                        Radices rz, const V* twy, const V* twz, cudaStream_t s) {
  ClusterGeom q;
  if (!pass_b_cluster_geom(g.nz, g.My, g.Mz, sizeof(V), &q)) {
    set_error("y-z plane %d x %d too large for pass B (eight-CTA cluster)", g.My, g.Mz);
    return VIE_ERR_INVALID;
  }
  const size_t smem = pass_b_cluster_smem(g, q, sizeof(V));
  VIE_CUDA_TRY(cudaFuncSetAttribute(pass_b_cluster_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(g.Mx * q.cs), (unsigned)count);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)q.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  VIE_CUDA_TRY(cudaLaunchKernelEx(&cfg, pass_b_cluster_kernel<V>, pp, g, q, ry, rz, twy, twz));
  return VIE_OK;
}

// ---------------------------------------------------------------------------
// Split pass B for planes too large for one CTA (y first, three launches):
//   B1 the x-pass kernel run along y: lines (kx, l), l = c nz + z, of ny
//      values, zero-padded to My, forward FFT; output Y[kx][ky][l] (the
//      x-pass kernels' transposed store, grouped by kx: gsz = 3 nz);
//   B2 pass_bz_kernel: per (kx, ky) the 3 nz values of the three components,
//      forward FFT along z in registers, folded 3x3 spectral multiply,
//      inverse FFT along z, z < nz back in place;
//   B3 the inverse x-pass kernel run along y with a plain epilogue: inverse
//      FFT, crop to ny, back into the workspace slab work[kx][l ny + y].
// A B2 block takes one folded kxf, kBzCells consecutive folded kyf and all
// their images (kx, Mx - kx) x (ky, My - ky): four contiguous runs of Y,
// and each folded spectrum entry is read from memory once per block and
// serves up to 8 spectral cells (kz and Mz - kz lie in the same thread's
// line).  Threads (c, cell) transform one
// component's z-line; the multiply exchanges them through shared memory.
// ---------------------------------------------------------------------------
constexpr int kBzCells = 16;
constexpr int kBzThreads = 3 * 4 * kBzCells;

// NZ > 0 fixes nz at compile time (the zero padding is not loaded and the
// cropped outputs are dead code; the additions of the padding zeros stay,
// since IEEE arithmetic keeps x + 0); NZ = 0 reads it from g.
template <typename V, int MZ, int NZ>
__global__ void __launch_bounds__(kBzThreads, sizeof(V) == sizeof(float2) ? 4 : 1)
    pass_bz_kernel(const __grid_constant__ PassPtrs<V> pp, PassBGeom g, int tiles, const V* __restrict__ twzg) {
  if (skip_problem(pp)) return;
  constexpr int C4 = 4 * kBzCells;
  constexpr int KZ = MZ / 2 + 1;
  const int nz = NZ > 0 ? NZ : g.nz, nl3 = 3 * nz;
  const int pio = nl3 | 1;
  extern __shared__ unsigned char smem_raw[];
  long long* base = reinterpret_cast<long long*>(smem_raw);   // Y offset of each cell, -1: no cell
  int* flip = reinterpret_cast<int*>(base + C4);              // bit 0: kx > Mx - kx, bit 1: ky > My - ky
  V* twz = reinterpret_cast<V*>(flip + C4);
  V* Gs = twz + MZ;                          // [comp][kzf][j]: 6 KZ kBzCells
  V* S = Gs + (size_t)6 * KZ * kBzCells;     // [c][kz][cell]
  V* IO = S;                                 // [cell][pio], shares S (pio <= 3 MZ)
  const int kxf = blockIdx.x / tiles;
  const int kyf0 = (blockIdx.x - kxf * tiles) * kBzCells;
  const int tid = threadIdx.x, nth = blockDim.x;
  pdl_launch_dependents();
  // plan constants before the dependency wait: twiddles and the spectrum tile
  for (int i = tid; i < MZ; i += nth) __pipeline_memcpy_async(twz + i, twzg + i, sizeof(V));
  {
    const V* G = pp.ghat[blockIdx.y] + (size_t)kxf * 6 * KZ * g.Ky;
    const int nj = min(kBzCells, g.Ky - kyf0);
    for (int e = tid; e < 6 * KZ * kBzCells; e += nth) {
      const int row = e / kBzCells, j = e - row * kBzCells;   // row = comp KZ + kzf
      if (j < nj) __pipeline_memcpy_async(Gs + e, G + (size_t)row * g.Ky + kyf0 + j, sizeof(V));
    }
  }
  __pipeline_commit();
  // cell = image * kBzCells + j: (kx, ky) = (kxf or Mx - kxf, kyf or My - kyf);
  // no cell where an image repeats another (kxf = 0 or Mx / 2, same for y)
  // or kyf lies past the folded range
  if (tid < C4) {
    const int img = tid / kBzCells, kyf = kyf0 + (tid - img * kBzCells);
    bool ok = kyf < g.Ky;
    if ((img & 1) && (kxf == 0 || 2 * kxf == g.Mx)) ok = false;
    if ((img & 2) && (kyf == 0 || 2 * kyf == g.My)) ok = false;
    const int kx = (img & 1) ? g.Mx - kxf : kxf;
    const int ky = (img & 2) ? g.My - kyf : kyf;
    base[tid] = ok ? ((long long)kx * g.My + ky) * nl3 : -1;
    flip[tid] = (kx > g.Mx - kx ? 1 : 0) | (ky > g.My - ky ? 2 : 0);
  }
  __syncthreads();
  pdl_wait();
  V* __restrict__ Y = pp.work2[blockIdx.y];
  for (int e = tid; e < C4 * nl3; e += nth) {   // all loads in flight at once
    const int cell = e / nl3, l = e - cell * nl3;
    const long long b = base[cell];
    if (b >= 0) __pipeline_memcpy_async(IO + cell * pio + l, Y + b + l, sizeof(V));
  }
  __pipeline_commit();
  __pipeline_wait_prior(0);
  __syncthreads();
  const int c = tid / C4, cell = tid - c * C4;
  const bool valid = base[cell] >= 0;
  {
    V a[MZ];
#pragma unroll
    for (int z = 0; z < MZ; ++z) a[z] = (valid && z < nz) ? IO[cell * pio + c * nz + z] : zero_c<V>();
    __syncthreads();   // every thread has its line: S may overwrite IO
    reg_fft<V, false, MZ>(a, twz);
#pragma unroll
    for (int kz = 0; kz < MZ; ++kz) S[(c * MZ + kz) * C4 + cell] = a[kz];
  }
  __syncthreads();
  // u_p = sum_q G_pq w_q: item (image, kzf, j) serves kz = kzf and Mz - kzf
  const int gcs = KZ * kBzCells;
  for (int e = tid; e < 4 * KZ * kBzCells; e += nth) {
    const int j = e % kBzCells, r = e / kBzCells;
    const int kzf = r % KZ, img = r / KZ;
    const int cl = img * kBzCells + j;
    if (base[cl] < 0) continue;
    const int fl = flip[cl];
    const bool fx = fl & 1, fy = fl & 2;
    const V* Gc = Gs + kzf * kBzCells + j;
    const V gxx = Gc[0], gyy = Gc[gcs], gzz = Gc[2 * gcs];
    const V gxy0 = Gc[3 * gcs], gxz0 = Gc[4 * gcs], gyz0 = Gc[5 * gcs];
    const int nkz = (kzf == 0 || 2 * kzf == MZ) ? 1 : 2;
    for (int t = 0; t < nkz; ++t) {
      const int kz = t ? MZ - kzf : kzf;
      const bool fz = t == 1;
      const V gxy = (fx ^ fy) ? scale(gxy0, -1.0f) : gxy0;
      const V gxz = (fx ^ fz) ? scale(gxz0, -1.0f) : gxz0;
      const V gyz = (fy ^ fz) ? scale(gyz0, -1.0f) : gyz0;
      V* px = S + (0 * MZ + kz) * C4 + cl;
      V* pyv = S + (1 * MZ + kz) * C4 + cl;
      V* pzv = S + (2 * MZ + kz) * C4 + cl;
      const V wx = *px, wy = *pyv, wz = *pzv;
      *px = add(add(mul(gxx, wx), mul(gxy, wy)), mul(gxz, wz));
      *pyv = add(add(mul(gxy, wx), mul(gyy, wy)), mul(gyz, wz));
      *pzv = add(add(mul(gxz, wx), mul(gyz, wy)), mul(gzz, wz));
    }
  }
  __syncthreads();
  {
    V a[MZ];
#pragma unroll
    for (int kz = 0; kz < MZ; ++kz) a[kz] = S[(c * MZ + kz) * C4 + cell];
    __syncthreads();   // every thread has its line: IO may overwrite S
    reg_fft<V, true, MZ>(a, twz);
#pragma unroll
    for (int z = 0; z < MZ; ++z)
      if (z < nz) IO[cell * pio + c * nz + z] = a[z];
  }
  __syncthreads();
  for (int e = tid; e < C4 * nl3; e += nth) {
    const int cell2 = e / nl3, l = e - cell2 * nl3;
    const long long b = base[cell2];
    if (b >= 0) Y[b + l] = IO[cell2 * pio + l];
  }
}

// z lengths with a compiled B2 kernel; other lengths use the cluster pass.
// (MZ, NZ) pairs with nz fixed at compile time: 220 nm layers at 20 nm.
#define VIE_PASS_BZ_SIZES(X) \
  X(4) X(5) X(6) X(8) X(9) X(10) X(12) X(15) X(16) X(18) X(20) X(24) X(25) X(27) X(30) X(32)
#define VIE_PASS_BZ_FIXED(X) X(24, 11) X(24, 12)

static bool pass_bz_available(int mz) {
#define VIE_X(a) if (mz == a) return true;
  VIE_PASS_BZ_SIZES(VIE_X)
#undef VIE_X
  return false;
}

template <typename V, int MZ, int NZ>
static vie_status launch_pass_bz(const PassPtrs<V>& pp, int count, const PassBGeom& g, const V* twz,
                                 cudaStream_t s) {
  constexpr int C4 = 4 * kBzCells;
  const int pio = (3 * g.nz) | 1;
  if (pio > 3 * MZ) { set_error("pass B2: nz = %d too large for Mz = %d", g.nz, MZ); return VIE_ERR_INVALID; }
  const size_t smem = (size_t)C4 * (sizeof(long long) + sizeof(int)) +
                      ((size_t)MZ + 6 * (size_t)(MZ / 2 + 1) * kBzCells + 3 * MZ * C4) * sizeof(V);
  if (smem > 220 * 1024) { set_error("pass B2 shared memory %zu too large", smem); return VIE_ERR_INVALID; }
  VIE_CUDA_TRY(cudaFuncSetAttribute(pass_bz_kernel<V, MZ, NZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  const int tiles = (g.Ky + kBzCells - 1) / kBzCells;
  const int Kx = g.Mx / 2 + 1;
  VIE_CUDA_TRY(launch_pdl(pass_bz_kernel<V, MZ, NZ>, dim3((unsigned)(Kx * tiles), (unsigned)count), dim3(kBzThreads),
                          smem, s, pp, g, tiles, twz));
  return VIE_OK;
}

template <typename V>
static vie_status dispatch_pass_bz(const PassPtrs<V>& pp, int count, const PassBGeom& g, const V* twz,
                                   cudaStream_t s) {
#define VIE_Y(a, b) if (g.Mz == a && g.nz == b) return launch_pass_bz<V, a, b>(pp, count, g, twz, s);
  VIE_PASS_BZ_FIXED(VIE_Y)
#undef VIE_Y
#define VIE_X(a) if (g.Mz == a) return launch_pass_bz<V, a, 0>(pp, count, g, twz, s);
  VIE_PASS_BZ_SIZES(VIE_X)
#undef VIE_X
  set_error("no z-stage kernel for Mz = %d", g.Mz);
  return VIE_ERR_INVALID;
}

// ---------------------------------------------------------------------------
// pass B with register FFTs for compile-time lengths (MY, MZ): one line per
// thread, four barriers per plane.  Shared rows use odd pitches so that
// threads walking their own rows hit distinct banks.
//   S1: (c, kz) y-lines, pitch PY;  S2: (c, y) z-lines, pitch PZ.
// ---------------------------------------------------------------------------
// NY, NZ > 0 fix the cross-section at compile time: the zero padding is not
// loaded and the cropped outputs are dead code (the first-stage additions of
// the padding zeros stay: IEEE arithmetic keeps x + 0).
template <typename V, int MY, int MZ, int NY, int NZ>
__global__ void __launch_bounds__(256) pass_b_reg_kernel(const __grid_constant__ PassPtrs<V> pp, PassBGeom g,
                                                         const V* __restrict__ twyg, const V* __restrict__ twzg) {
  if (skip_problem(pp)) return;
  V* __restrict__ work = pp.work[blockIdx.y];
  const V* __restrict__ ghat = pp.ghat[blockIdx.y];
  constexpr int PY = (MY % 2 == 0) ? MY + 1 : MY;
  constexpr int PZ = (MZ % 2 == 0) ? MZ + 1 : MZ;
  extern __shared__ unsigned char smem_raw[];
  V* twy = reinterpret_cast<V*>(smem_raw);
  V* twz = twy + MY;
  V* S1 = twz + MZ;
  V* S2 = S1 + 3 * MZ * PY;
  V* Gs = S2 + 3 * g.ny * PZ;          // folded spectrum chunk of this kx, 6 Kz Ky
  const int kx = blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int ny = NY > 0 ? NY : g.ny, nz = NZ > 0 ? NZ : g.nz;
  const bool fx = kx > g.Mx - kx;
  const int kxf = fx ? g.Mx - kx : kx;
  pdl_launch_dependents();
  // plan constants first (allowed before the dependency wait)
  for (int i = tid; i < MY; i += nth) __pipeline_memcpy_async(twy + i, twyg + i, sizeof(V));
  for (int i = tid; i < MZ; i += nth) __pipeline_memcpy_async(twz + i, twzg + i, sizeof(V));
  __pipeline_commit();
  {
    // spectrum chunk: lands while the z and y transforms run
    const V* G = ghat + (size_t)kxf * 6 * g.Kz * g.Ky;
    const int chunk = 6 * g.Kz * g.Ky;
    for (int i = tid; i < chunk; i += nth) __pipeline_memcpy_async(Gs + i, G + i, sizeof(V));
    __pipeline_commit();
  }
  pdl_wait();                 // the x pass that wrote the slab has completed
  __pipeline_wait_prior(1);   // twiddles done; the spectrum may still be in flight
  __syncthreads();
  V* slab = work + (size_t)kx * g.NL;
  // forward z on the 3 ny non-zero lines (c, y)
  for (int line = tid; line < 3 * ny; line += nth) {
    const int c = line / ny, y = line - c * ny;
    V a[MZ];
#pragma unroll
    for (int z = 0; z < MZ; ++z) a[z] = (z < nz) ? slab[(c * nz + z) * ny + y] : zero_c<V>();
    reg_fft<V, false, MZ>(a, twz);
#pragma unroll
    for (int kz = 0; kz < MZ; ++kz) S1[(c * MZ + kz) * PY + y] = a[kz];
  }
  __syncthreads();
  // forward y on all 3 MZ lines (c, kz); y >= ny is zero padding
  for (int line = tid; line < 3 * MZ; line += nth) {
    V a[MY];
#pragma unroll
    for (int y = 0; y < MY; ++y) a[y] = (y < ny) ? S1[line * PY + y] : zero_c<V>();
    reg_fft<V, false, MY>(a, twy);
#pragma unroll
    for (int ky = 0; ky < MY; ++ky) S1[line * PY + ky] = a[ky];
  }
  __pipeline_wait_prior(0);
  __syncthreads();
  {
    const V* G = Gs;
    const int cs = g.Kz * g.Ky;
    for (int e = tid; e < MZ * MY; e += nth) {
      const int kz = e / MY, ky = e - kz * MY;
      const bool fy = ky > MY - ky, fz = kz > MZ - kz;
      const int kyf = fy ? MY - ky : ky, kzf = fz ? MZ - kz : kz;
      const size_t o = (size_t)kzf * g.Ky + kyf;
      V gxx = G[o], gyy = G[cs + o], gzz = G[2 * cs + o];
      V gxy = G[3 * cs + o], gxz = G[4 * cs + o], gyz = G[5 * cs + o];
      if (fx ^ fy) gxy = scale(gxy, -1.0f);
      if (fx ^ fz) gxz = scale(gxz, -1.0f);
      if (fy ^ fz) gyz = scale(gyz, -1.0f);
      V* px = S1 + (0 * MZ + kz) * PY + ky;
      V* pyv = S1 + (1 * MZ + kz) * PY + ky;
      V* pzv = S1 + (2 * MZ + kz) * PY + ky;
      const V wx = *px, wy = *pyv, wz = *pzv;
      *px = add(add(mul(gxx, wx), mul(gxy, wy)), mul(gxz, wz));
      *pyv = add(add(mul(gxy, wx), mul(gyy, wy)), mul(gyz, wz));
      *pzv = add(add(mul(gxz, wx), mul(gyz, wy)), mul(gzz, wz));
    }
  }
  __syncthreads();
  // inverse y; keep y < ny, stored as z-lines (c, y)
  for (int line = tid; line < 3 * MZ; line += nth) {
    const int c = line / MZ, kz = line - c * MZ;
    V a[MY];
#pragma unroll
    for (int ky = 0; ky < MY; ++ky) a[ky] = S1[line * PY + ky];
    reg_fft<V, true, MY>(a, twy);
#pragma unroll
    for (int y = 0; y < MY; ++y)
      if (y < ny) S2[(c * ny + y) * PZ + kz] = a[y];
  }
  __syncthreads();
  // inverse z; keep z < nz, back to the workspace slab
  for (int line = tid; line < 3 * ny; line += nth) {
    const int c = line / ny, y = line - c * ny;
    V a[MZ];
#pragma unroll
    for (int kz = 0; kz < MZ; ++kz) a[kz] = S2[line * PZ + kz];
    reg_fft<V, true, MZ>(a, twz);
#pragma unroll
    for (int z = 0; z < MZ; ++z)
      if (z < nz) slab[(c * nz + z) * ny + y] = a[z];
  }
}

// (MY, MZ) pairs with a register-FFT pass B; other sizes use pass_b_kernel.
#define VIE_PASS_B_REG_SIZES(X) \
  X(24, 24) X(45, 24) X(48, 24) X(50, 24) X(30, 24) X(40, 24) X(25, 24) X(45, 25) X(48, 25) X(24, 25)
// (MY, MZ, NY, NZ) with the cross-section compiled in: the 460 x 220 nm strip
// at 20 nm (23 x 11 voxels) in its smallest 5-smooth embeddings.
#define VIE_PASS_B_REG_FIXED(X) X(45, 24, 23, 11) X(48, 24, 23, 11)

bool pass_b_reg_available(int my, int mz) {
#define VIE_X(a, b) if (my == a && mz == b) return true;
  VIE_PASS_B_REG_SIZES(VIE_X)
#undef VIE_X
  return false;
}

template <typename V, int MY, int MZ, int NY, int NZ>
static vie_status launch_pass_b_reg(const PassPtrs<V>& pp, int count, const PassBGeom& g, const V* twy,
                                    const V* twz, cudaStream_t s) {
  constexpr int PY = (MY % 2 == 0) ? MY + 1 : MY;
  constexpr int PZ = (MZ % 2 == 0) ? MZ + 1 : MZ;
  const size_t smem = (size_t)(MY + MZ + 3 * MZ * PY + 3 * g.ny * PZ + 6 * g.Kz * g.Ky) * sizeof(V);
  if (smem > 220 * 1024) { set_error("pass B shared memory %zu too large", smem); return VIE_ERR_INVALID; }
  VIE_CUDA_TRY(cudaFuncSetAttribute(pass_b_reg_kernel<V, MY, MZ, NY, NZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  int lines = 3 * (g.ny > MZ ? g.ny : MZ);
  int threads = ((lines + 31) / 32) * 32;
  if (threads > 256) threads = 256;
  VIE_CUDA_TRY(launch_pdl(pass_b_reg_kernel<V, MY, MZ, NY, NZ>, dim3((unsigned)g.Mx, (unsigned)count), dim3(threads), smem,
                          s, pp, g, twy, twz));
  return VIE_OK;
}

// complex128 lines longer than 30 would spill registers: those keep the generic pass
template <typename V, int MY, int MZ, int NY = 0, int NZ = 0>
static vie_status try_pass_b_reg(const PassPtrs<V>& pp, int count, const PassBGeom& g, const V* twy,
                                 const V* twz, cudaStream_t s, bool* done) {
  if constexpr (sizeof(V) == sizeof(float2) || (MY <= 30 && MZ <= 30)) {
    *done = true;
    return launch_pass_b_reg<V, MY, MZ, NY, NZ>(pp, count, g, twy, twz, s);
  } else {
    *done = false;
    return VIE_OK;
  }
}

template <typename V>
static vie_status dispatch_pass_b_reg(const PassPtrs<V>& pp, int count, const PassBGeom& g, const V* twy,
                                      const V* twz, cudaStream_t s, bool* done) {
  *done = false;
#define VIE_X(a, b) \
  if (g.My == a && g.Mz == b) return try_pass_b_reg<V, a, b>(pp, count, g, twy, twz, s, done);
#define VIE_Y(a, b, c, d)                       \
  if (g.My == a && g.Mz == b && g.ny == c && g.nz == d) \
    return try_pass_b_reg<V, a, b, c, d>(pp, count, g, twy, twz, s, done);
  VIE_PASS_B_REG_FIXED(VIE_Y)
#undef VIE_Y
  VIE_PASS_B_REG_SIZES(VIE_X)
#undef VIE_X
  return VIE_OK;
}

// ---------------------------------------------------------------------------
// pass C
// ---------------------------------------------------------------------------
template <typename V>
__global__ void __launch_bounds__(256) pass_c_kernel(const __grid_constant__ PassPtrs<V> pp, int nx, int nyz,
                                                     int NL, Radices rx, const V* __restrict__ twg,
                                                     int lines_per_block, int mode, int gsz) {
  if (skip_problem(pp)) return;
  pdl_wait();
  const V* __restrict__ work = pp.work[blockIdx.y];
  const V* __restrict__ x = pp.x[blockIdx.y];
  const V* __restrict__ Mc = pp.M[blockIdx.y];
  V* __restrict__ y = pp.y[blockIdx.y];
  extern __shared__ unsigned char smem_raw[];
  const int Mx = rx.len;
  const int pitch = Mx + 1;
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* A = tw + Mx;
  V* B = A + (size_t)lines_per_block * pitch;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int l0 = blockIdx.x * lines_per_block;
  const int nl = min(lines_per_block, NL - l0);
  for (int i = tid; i < Mx; i += nth) tw[i] = twg[i];
  for (int e = tid; e < nl * Mx; e += nth) {
    const int kx = e / nl, l = e - kx * nl;
    const int line = l0 + l, grp = line / gsz;
    A[l * pitch + kx] = work[((size_t)grp * Mx + kx) * gsz + (line - grp * gsz)];
  }
  __syncthreads();
  V* res = fft_lines<V, true>(A, B, rx, pitch, nl, tw, tid, nth);
  for (int e = tid; e < nl * nx; e += nth) {
    const int l = e / nx, ix = e - l * nx;
    const int line = l0 + l;
    const size_t gi = (size_t)line * nx + ix;
    const size_t vox = (size_t)(line % nyz) * nx + ix;
    const V u = res[l * pitch + ix];
    if (mode == MODE_PLAIN) { y[gi] = u; continue; }
    const V w = x[gi];
    const V m = Mc[vox];
    y[gi] = (mode == MODE_OPERATOR) ? sub(w, mul(m, u)) : mul(m, sub(u, w));
  }
}

// ---------------------------------------------------------------------------
// x passes with a four-step register FFT, Mx = L1 * L2 (compile time).
// Index maps: input n = n1 + L1 n2, output k = k2 + L2 k1.
//   step 1: thread (l, n1) transforms the L2 values n1 + L1 n2 and multiplies by
//           w_Mx^(n1 k2);  step 2: thread (l, k2) transforms the L1 values.
// Lanes run fastest over the LPB lines of the block, so the transposed
// workspace accesses work[k][line] are contiguous across a warp.  Lines may
// be grouped (gsz lines per group, work[group][k][line in group]); the x
// passes use one group (gsz = NL).  Shared rows
// are padded to a pitch congruent to LPB mod 16 (no bank conflicts for 8-byte
// elements).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int pitch_mod16(int n, int lpb) { return n + ((lpb - n % 16) % 16 + 16) % 16; }

// NX > 0 (a multiple of L1 for pass A, of L2 for pass C) fixes the line
// length at compile time: the zero padding of the forward transform is not
// loaded and the cropped outputs of the inverse are dead code (the additions
// of the padding zeros stay: IEEE arithmetic keeps x + 0).
template <typename V, int L1, int L2, int LPB, int NX>
__global__ void __launch_bounds__(LPB * (L1 > L2 ? L1 : L2)) pass_a4_kernel(
    const __grid_constant__ PassPtrs<V> pp, int nx, int NL, const V* __restrict__ twxg, int gsz) {
  if (skip_problem(pp)) return;
  static_assert(NX == 0 || (NX % L1 == 0 && NX % L2 == 0), "compiled line length must divide by L1 and L2");
  const V* __restrict__ x = pp.x[blockIdx.y];
  V* __restrict__ work = pp.work[blockIdx.y];
  constexpr int MX = L1 * L2;
  constexpr int R = pitch_mod16(L1 * LPB, LPB);
  extern __shared__ unsigned char smem_raw[];
  V* twx = reinterpret_cast<V*>(smem_raw);
  V* tw1 = twx + MX;
  V* tw2 = tw1 + L1;
  V* T = tw2 + L2;                 // [k2][R], element (n1, l) at n1 * LPB + l
  V* Xs = T + L2 * R;              // [l][P]
  const int P = pitch_mod16(nx, LPB);
  const int tid = threadIdx.x, nth = blockDim.x;
  const int l0 = blockIdx.x * LPB;
  const int nl = min(LPB, NL - l0);
  pdl_launch_dependents();
  {
    // asynchronous copies of the twiddles (plan constants) and, once the
    // producer of x is done, of the block's lines (contiguous in x)
    for (int i = tid; i < MX; i += nth) __pipeline_memcpy_async(twx + i, twxg + i, sizeof(V));
    pdl_wait();
    const V* src = x + (size_t)l0 * nx;
    for (int l = 0; l < nl; ++l)
      for (int n = tid; n < nx; n += nth) __pipeline_memcpy_async(Xs + l * P + n, src + (size_t)l * nx + n, sizeof(V));
    __pipeline_commit();
    __pipeline_wait_prior(0);
  }
  __syncthreads();
  for (int i = tid; i < L1; i += nth) tw1[i] = twx[i * L2];   // w_L1^i = w_Mx^(i L2)
  for (int i = tid; i < L2; i += nth) tw2[i] = twx[i * L1];
  __syncthreads();
  if (tid < LPB * L1) {
    const int l = tid % LPB, n1 = tid / LPB;
    V a[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) {
      const int n = n1 + L1 * n2;
      const bool in = NX > 0 ? (n2 < NX / L1) : (n < nx);
      a[n2] = (l < nl && in) ? Xs[l * P + n] : zero_c<V>();
    }
    reg_fft<V, false, L2>(a, tw2);
#pragma unroll
    for (int k2 = 0; k2 < L2; ++k2) T[k2 * R + n1 * LPB + l] = (k2 == 0) ? a[0] : mul(a[k2], twx[n1 * k2]);
  }
  __syncthreads();
  if (tid < LPB * L2) {
    const int l = tid % LPB, k2 = tid / LPB;
    V a[L1];
#pragma unroll
    for (int n1 = 0; n1 < L1; ++n1) a[n1] = T[k2 * R + n1 * LPB + l];
    reg_fft<V, false, L1>(a, tw1);
    if (l < nl) {
      const int line = l0 + l, grp = line / gsz;
      V* dst = work + (size_t)grp * MX * gsz + (line - grp * gsz);
#pragma unroll
      for (int k1 = 0; k1 < L1; ++k1) dst[(size_t)(k2 + L2 * k1) * gsz] = a[k1];
    }
  }
}

template <typename V, int L1, int L2, int LPB, int NX>
__global__ void __launch_bounds__(LPB * (L1 > L2 ? L1 : L2)) pass_c4_kernel(
    const __grid_constant__ PassPtrs<V> pp, int nx, int nyz, int NL, const V* __restrict__ twxg, int mode,
    int gsz) {
  if (skip_problem(pp)) return;
  const V* __restrict__ work = pp.work[blockIdx.y];
  const V* __restrict__ x = pp.x[blockIdx.y];
  const V* __restrict__ Mc = pp.M[blockIdx.y];
  V* __restrict__ y = pp.y[blockIdx.y];
  constexpr int MX = L1 * L2;
  constexpr int R = pitch_mod16(L1 * LPB, LPB);
  extern __shared__ unsigned char smem_raw[];
  V* twx = reinterpret_cast<V*>(smem_raw);
  V* tw1 = twx + MX;
  V* tw2 = tw1 + L1;
  V* T = tw2 + L2;
  V* Ys = T + L2 * R;
  const int P = pitch_mod16(nx, LPB);
  V* Xs = Ys + LPB * P;            // the block's rows of x (epilogue operand)
  V* Ms = Xs + LPB * nx;           // the matching rows of M
  const int tid = threadIdx.x, nth = blockDim.x;
  const int l0 = blockIdx.x * LPB;
  const int nl = min(LPB, NL - l0);
  pdl_launch_dependents();
  {
    // asynchronous copies: twiddles now, epilogue operands to land during the
    // FFTs; the contrast rows are plan data, x only after the dependency wait
    for (int i = tid; i < MX; i += nth) __pipeline_memcpy_async(twx + i, twxg + i, sizeof(V));
    __pipeline_commit();
    if (mode != MODE_PLAIN) {
      for (int l = 0; l < nl; ++l) {
        const V* msrc = Mc + (size_t)((l0 + l) % nyz) * nx;
        for (int i = tid; i < nx; i += nth) __pipeline_memcpy_async(Ms + l * nx + i, msrc + i, sizeof(V));
      }
    }
    pdl_wait();
    if (mode != MODE_PLAIN) {
      const V* xsrc = x + (size_t)l0 * nx;
      for (int e = tid; e < nl * nx; e += nth) __pipeline_memcpy_async(Xs + e, xsrc + e, sizeof(V));
    }
    __pipeline_commit();
    __pipeline_wait_prior(1);      // twiddles only
  }
  __syncthreads();
  for (int i = tid; i < L1; i += nth) tw1[i] = twx[i * L2];   // w_L1^i = w_Mx^(i L2)
  for (int i = tid; i < L2; i += nth) tw2[i] = twx[i * L1];
  __syncthreads();
  // inverse transform, same decomposition with conjugate twiddles:
  // input a = a1 + L1 a2 (a spectrum index kx), output b = b2 + L2 b1 (x)
  if (tid < LPB * L1) {
    const int l = tid % LPB, a1 = tid / LPB;
    const int line = l0 + (l < nl ? l : 0), grp = line / gsz;
    const V* src = work + (size_t)grp * MX * gsz + (line - grp * gsz);
    V a[L2];
#pragma unroll
    for (int a2 = 0; a2 < L2; ++a2) a[a2] = (l < nl) ? src[(size_t)(a1 + L1 * a2) * gsz] : zero_c<V>();
    reg_fft<V, true, L2>(a, tw2);
#pragma unroll
    for (int b2 = 0; b2 < L2; ++b2) T[b2 * R + a1 * LPB + l] = (b2 == 0) ? a[0] : mulc(a[b2], twx[a1 * b2]);
  }
  __syncthreads();
  if (tid < LPB * L2) {
    const int l = tid % LPB, b2 = tid / LPB;
    V a[L1];
#pragma unroll
    for (int a1 = 0; a1 < L1; ++a1) a[a1] = T[b2 * R + a1 * LPB + l];
    reg_fft<V, true, L1>(a, tw1);
#pragma unroll
    for (int b1 = 0; b1 < L1; ++b1) {
      const int n = b2 + L2 * b1;
      if (NX > 0 ? (b1 < NX / L2) : (n < nx)) Ys[l * P + n] = a[b1];
    }
  }
  __syncthreads();
  __pipeline_wait_prior(0);
  __syncthreads();
  {
    // contrast epilogue from the prefetched rows
    const int total = nl * nx;
    const size_t g0 = (size_t)l0 * nx;
    for (int e = tid; e < total; e += nth) {
      const int l = e / nx, ix = e - l * nx;
      const V uu = Ys[l * P + ix];
      if (mode == MODE_PLAIN) { y[g0 + e] = uu; continue; }
      const V wv = Xs[e], mv = Ms[e];
      y[g0 + e] = (mode == MODE_OPERATOR) ? sub(wv, mul(mv, uu)) : mul(mv, sub(uu, wv));
    }
  }
}

// ---------------------------------------------------------------------------
// x passes with a three-factor register FFT, Mx = L1 L2 L3 (compile time),
// for lines too few to keep the SMs busy with one thread per sub-FFT of the
// four-step split (759 lines of the 600 x 23 x 11 guide give 30k threads at
// Mx = 40 x 30, six warps per SM).  Index maps (M = L2 L3):
//   input  n  = n1 + L1 (m2 + L2 m3),  output k = kM + M k1, kM = k3 + L3 k2;
//   step 1: thread (l, n1, m2) transforms the L3 values over m3 and multiplies
//           by w_M^(m2 k3) = w_Mx^(L1 m2 k3);
//   step 2: thread (l, n1, k3) transforms the L2 values over m2 and multiplies
//           by w_Mx^(n1 kM);
//   step 3: thread (l, kM) transforms the L1 values over n1.
// LPB lines per block, lanes fastest over the lines.  NX > 0 fixes the line
// length: the forward pass drops m3 >= NX / (L1 L2) (zero padding) and the
// inverse pass keeps k1 < NX / M (the crop).  The inverse pass runs the same
// steps with conjugate twiddles on spectrum index n (the workspace) and
// spatial index k, then applies the contrast epilogue.
// ---------------------------------------------------------------------------
template <int L1, int L2, int L3>
struct X3 {
  static constexpr int MX = L1 * L2 * L3;
  static constexpr int M = L2 * L3;
  static constexpr int T1 = L1 * L2, T2 = L1 * L3, T3 = L2 * L3;
  static constexpr int NT = (T1 > T2 ? (T1 > T3 ? T1 : T3) : (T2 > T3 ? T2 : T3));
};

template <typename V, int L1, int L2, int L3, int LPB, bool INV>
__device__ __forceinline__ void x3_steps12(V* __restrict__ S1, V* __restrict__ S2, const V* __restrict__ twx,
                                           const V* __restrict__ tw2, const V* __restrict__ tw3, int R1, int R2,
                                           V (&a)[L3], int tid) {
  typedef X3<L1, L2, L3> G;
  // step 1 (a holds this thread's L3 inputs over m3)
  if (tid < LPB * G::T1) {
    const int l = tid % LPB, r = tid / LPB;           // r = n1 + L1 m2
    const int m2 = r / L1;
    reg_fft<V, INV, L3>(a, tw3);
#pragma unroll
    for (int k3 = 0; k3 < L3; ++k3) {
      const V t = (k3 == 0 || m2 == 0) ? a[k3] : (INV ? mulc(a[k3], twx[L1 * m2 * k3]) : mul(a[k3], twx[L1 * m2 * k3]));
      S1[k3 * R1 + r * LPB + l] = t;
    }
  }
  __syncthreads();
  // step 2
  if (tid < LPB * G::T2) {
    const int l = tid % LPB, r = tid / LPB;           // r = n1 + L1 k3
    const int n1 = r % L1, k3 = r / L1;
    V b[L2];
#pragma unroll
    for (int m2 = 0; m2 < L2; ++m2) b[m2] = S1[k3 * R1 + (n1 + L1 * m2) * LPB + l];
    reg_fft<V, INV, L2>(b, tw2);
#pragma unroll
    for (int k2 = 0; k2 < L2; ++k2) {
      const int kM = k3 + L3 * k2;
      const V t = (n1 == 0 || kM == 0) ? b[k2] : (INV ? mulc(b[k2], twx[n1 * kM]) : mul(b[k2], twx[n1 * kM]));
      S2[kM * R2 + n1 * LPB + l] = t;
    }
  }
  __syncthreads();
}

template <typename V, int L1, int L2, int L3, int LPB, int NX>
__global__ void __launch_bounds__(LPB * X3<L1, L2, L3>::NT) pass_a3_kernel(
    const __grid_constant__ PassPtrs<V> pp, int nx, int NL, const V* __restrict__ twxg, int gsz) {
  if (skip_problem(pp)) return;
  typedef X3<L1, L2, L3> G;
  static_assert(NX == 0 || NX % (L1 * L2) == 0, "compiled line length must divide by L1 L2");
  const V* __restrict__ x = pp.x[blockIdx.y];
  V* __restrict__ work = pp.work[blockIdx.y];
  constexpr int R1 = pitch_mod16(G::T1 * LPB, LPB);
  constexpr int R2 = pitch_mod16(L1 * LPB, LPB);
  extern __shared__ unsigned char smem_raw[];
  V* twx = reinterpret_cast<V*>(smem_raw);
  V* tw1 = twx + G::MX;
  V* tw2 = tw1 + L1;
  V* tw3 = tw2 + L2;
  V* S1 = tw3 + L3;                // [k3][R1]: (n1 + L1 m2, l)
  V* S2 = S1 + L3 * R1;            // [kM][R2]: (n1, l)
  V* Xs = S2 + G::M * R2;          // [l][P]
  const int P = pitch_mod16(nx, LPB);
  const int tid = threadIdx.x, nth = blockDim.x;
  const int l0 = blockIdx.x * LPB;
  const int nl = min(LPB, NL - l0);
  pdl_launch_dependents();
  {
    for (int i = tid; i < G::MX; i += nth) __pipeline_memcpy_async(twx + i, twxg + i, sizeof(V));
    pdl_wait();
    const V* src = x + (size_t)l0 * nx;
    for (int l = 0; l < nl; ++l)
      for (int n = tid; n < nx; n += nth) __pipeline_memcpy_async(Xs + l * P + n, src + (size_t)l * nx + n, sizeof(V));
    __pipeline_commit();
    __pipeline_wait_prior(0);
  }
  __syncthreads();
  for (int i = tid; i < L1; i += nth) tw1[i] = twx[i * (G::MX / L1)];
  for (int i = tid; i < L2; i += nth) tw2[i] = twx[i * (G::MX / L2)];
  for (int i = tid; i < L3; i += nth) tw3[i] = twx[i * (G::MX / L3)];
  __syncthreads();
  V a[L3];
  if (tid < LPB * G::T1) {
    const int l = tid % LPB, r = tid / LPB;
    const int n1 = r % L1, m2 = r / L1;
#pragma unroll
    for (int m3 = 0; m3 < L3; ++m3) {
      const int n = n1 + L1 * (m2 + L2 * m3);
      const bool in = NX > 0 ? (m3 < NX / (L1 * L2)) : (n < nx);
      a[m3] = (l < nl && in) ? Xs[l * P + n] : zero_c<V>();
    }
  }
  x3_steps12<V, L1, L2, L3, LPB, false>(S1, S2, twx, tw2, tw3, R1, R2, a, tid);
  // step 3: X[kM + M k1], written transposed (work[k][line])
  if (tid < LPB * G::T3) {
    const int l = tid % LPB, kM = tid / LPB;
    V c[L1];
#pragma unroll
    for (int n1 = 0; n1 < L1; ++n1) c[n1] = S2[kM * R2 + n1 * LPB + l];
    reg_fft<V, false, L1>(c, tw1);
    if (l < nl) {
      const int line = l0 + l, grp = line / gsz;
      V* dst = work + (size_t)grp * G::MX * gsz + (line - grp * gsz);
#pragma unroll
      for (int k1 = 0; k1 < L1; ++k1) dst[(size_t)(kM + G::M * k1) * gsz] = c[k1];
    }
  }
}

template <typename V, int L1, int L2, int L3, int LPB, int NX>
__global__ void __launch_bounds__(LPB * X3<L1, L2, L3>::NT) pass_c3_kernel(
    const __grid_constant__ PassPtrs<V> pp, int nx, int nyz, int NL, const V* __restrict__ twxg, int mode,
    int gsz) {
  if (skip_problem(pp)) return;
  typedef X3<L1, L2, L3> G;
  static_assert(NX == 0 || NX % G::M == 0, "compiled line length must divide by L2 L3");
  const V* __restrict__ work = pp.work[blockIdx.y];
  const V* __restrict__ x = pp.x[blockIdx.y];
  const V* __restrict__ Mc = pp.M[blockIdx.y];
  V* __restrict__ y = pp.y[blockIdx.y];
  constexpr int R1 = pitch_mod16(G::T1 * LPB, LPB);
  constexpr int R2 = pitch_mod16(L1 * LPB, LPB);
  extern __shared__ unsigned char smem_raw[];
  V* twx = reinterpret_cast<V*>(smem_raw);
  V* tw1 = twx + G::MX;
  V* tw2 = tw1 + L1;
  V* tw3 = tw2 + L2;
  V* S1 = tw3 + L3;
  V* S2 = S1 + L3 * R1;
  V* Ys = S2 + G::M * R2;          // [l][P] the inverse transform, x < nx
  const int P = pitch_mod16(nx, LPB);
  V* Xs = Ys + LPB * P;            // the block's rows of x (epilogue operand)
  V* Ms = Xs + LPB * nx;           // the matching rows of M
  const int tid = threadIdx.x, nth = blockDim.x;
  const int l0 = blockIdx.x * LPB;
  const int nl = min(LPB, NL - l0);
  pdl_launch_dependents();
  {
    for (int i = tid; i < G::MX; i += nth) __pipeline_memcpy_async(twx + i, twxg + i, sizeof(V));
    __pipeline_commit();
    if (mode != MODE_PLAIN) {
      for (int l = 0; l < nl; ++l) {
        const V* msrc = Mc + (size_t)((l0 + l) % nyz) * nx;
        for (int i = tid; i < nx; i += nth) __pipeline_memcpy_async(Ms + l * nx + i, msrc + i, sizeof(V));
      }
    }
    pdl_wait();
    if (mode != MODE_PLAIN) {
      const V* xsrc = x + (size_t)l0 * nx;
      for (int e = tid; e < nl * nx; e += nth) __pipeline_memcpy_async(Xs + e, xsrc + e, sizeof(V));
    }
    __pipeline_commit();
    __pipeline_wait_prior(1);      // twiddles only
  }
  __syncthreads();
  for (int i = tid; i < L1; i += nth) tw1[i] = twx[i * (G::MX / L1)];
  for (int i = tid; i < L2; i += nth) tw2[i] = twx[i * (G::MX / L2)];
  for (int i = tid; i < L3; i += nth) tw3[i] = twx[i * (G::MX / L3)];
  __syncthreads();
  V a[L3];
  if (tid < LPB * G::T1) {
    const int l = tid % LPB, r = tid / LPB;
    const int n1 = r % L1, m2 = r / L1;
    const int line = l0 + (l < nl ? l : 0), grp = line / gsz;
    const V* src = work + (size_t)grp * G::MX * gsz + (line - grp * gsz);
#pragma unroll
    for (int m3 = 0; m3 < L3; ++m3)
      a[m3] = (l < nl) ? src[(size_t)(n1 + L1 * (m2 + L2 * m3)) * gsz] : zero_c<V>();
  }
  x3_steps12<V, L1, L2, L3, LPB, true>(S1, S2, twx, tw2, tw3, R1, R2, a, tid);
  if (tid < LPB * G::T3) {
    const int l = tid % LPB, kM = tid / LPB;
    V c[L1];
#pragma unroll
    for (int n1 = 0; n1 < L1; ++n1) c[n1] = S2[kM * R2 + n1 * LPB + l];
    reg_fft<V, true, L1>(c, tw1);
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) {
      const int xo = kM + G::M * k1;
      if (NX > 0 ? (k1 < NX / G::M) : (xo < nx)) Ys[l * P + xo] = c[k1];
    }
  }
  __syncthreads();
  __pipeline_wait_prior(0);
  __syncthreads();
  {
    const int total = nl * nx;
    const size_t g0 = (size_t)l0 * nx;
    for (int e = tid; e < total; e += nth) {
      const int l = e / nx, ix = e - l * nx;
      const V uu = Ys[l * P + ix];
      if (mode == MODE_PLAIN) { y[g0 + e] = uu; continue; }
      const V wv = Xs[e], mv = Ms[e];
      y[g0 + e] = (mode == MODE_OPERATOR) ? sub(wv, mul(mv, uu)) : mul(mv, sub(uu, wv));
    }
  }
}

// Mx = L1 L2 L3 factorisations with a three-factor register x pass, and the
// compiled line lengths.
#define VIE_PASS_X3_SIZES(X) X(10, 12, 10)
#define VIE_PASS_X3_FIXED(X) X(10, 12, 10, 600)

template <typename V, int L1, int L2, int L3, int LPB, int NX>
static vie_status launch_x3_lpb(bool forward, const PassPtrs<V>& pp, int count, int nx, int nyz, int NL,
                                const V* twx, int mode, cudaStream_t s, bool* done, int gsz) {
  typedef X3<L1, L2, L3> G;
  constexpr int R1 = pitch_mod16(G::T1 * LPB, LPB);
  constexpr int R2 = pitch_mod16(L1 * LPB, LPB);
  const int P = pitch_mod16(nx, LPB);
  const bool operands = !forward && mode != MODE_PLAIN;
  const size_t smem = (size_t)(G::MX + L1 + L2 + L3 + L3 * R1 + G::M * R2 + LPB * P +
                               (forward ? 0 : (operands ? 2 * LPB * nx : 0))) * sizeof(V);
  if (smem > 200 * 1024) { *done = false; return VIE_OK; }
  const dim3 blocks((unsigned)((NL + LPB - 1) / LPB), (unsigned)count);
  const dim3 threads(LPB * G::NT);
  if (forward) {
    VIE_CUDA_TRY(cudaFuncSetAttribute(pass_a3_kernel<V, L1, L2, L3, LPB, NX>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    VIE_CUDA_TRY(launch_pdl(pass_a3_kernel<V, L1, L2, L3, LPB, NX>, blocks, threads, smem, s, pp, nx, NL, twx, gsz));
  } else {
    VIE_CUDA_TRY(cudaFuncSetAttribute(pass_c3_kernel<V, L1, L2, L3, LPB, NX>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    VIE_CUDA_TRY(launch_pdl(pass_c3_kernel<V, L1, L2, L3, LPB, NX>, blocks, threads, smem, s, pp, nx, nyz, NL, twx,
                            mode, gsz));
  }
  VIE_LAUNCH_CHECK();
  *done = true;
  return VIE_OK;
}

// lpb: 1, 2 or 5 lines per block (0: 5 where x_lines_five holds and the
// complex64 kernel with the line length compiled in exists, else 2)
template <typename V, int L1, int L2, int L3, int NX = 0>
static vie_status launch_x3(bool forward, const PassPtrs<V>& pp, int count, int nx, int nyz, int NL, const V* twx,
                            int mode, cudaStream_t s, bool* done, int lpb, int gsz) {
  if (lpb == 1) return launch_x3_lpb<V, L1, L2, L3, 1, NX>(forward, pp, count, nx, nyz, NL, twx, mode, s, done, gsz);
  if constexpr (sizeof(V) == sizeof(float2) && NX > 0) {
    if (lpb == 5 || (lpb == 0 && x_lines_five(NL, count)))
      return launch_x3_lpb<V, L1, L2, L3, 5, NX>(forward, pp, count, nx, nyz, NL, twx, mode, s, done, gsz);
  }
  return launch_x3_lpb<V, L1, L2, L3, 2, NX>(forward, pp, count, nx, nyz, NL, twx, mode, s, done, gsz);
}

// factors (L1, L2, L3) of Mx with a compiled three-factor kernel, or (0, 0, 0)
void x3_factors(int mx, int* l1, int* l2, int* l3) {
  *l1 = *l2 = *l3 = 0;
#define VIE_X(a, b, c) if (mx == a * b * c && *l1 == 0) { *l1 = a; *l2 = b; *l3 = c; }
  VIE_PASS_X3_SIZES(VIE_X)
#undef VIE_X
}

template <typename V>
static vie_status dispatch_x3(bool forward, int l1, int l2, int l3, const PassPtrs<V>& pp, int count, int nx,
                              int nyz, int NL, const V* twx, int mode, cudaStream_t s, bool* done, int lpb,
                              int gsz) {
  *done = false;
#define VIE_Y(a, b, c, d)                                        \
  if (l1 == a && l2 == b && l3 == c && nx == d)                   \
    return launch_x3<V, a, b, c, d>(forward, pp, count, nx, nyz, NL, twx, mode, s, done, lpb, gsz);
  VIE_PASS_X3_FIXED(VIE_Y)
#undef VIE_Y
#define VIE_X(a, b, c) \
  if (l1 == a && l2 == b && l3 == c) return launch_x3<V, a, b, c>(forward, pp, count, nx, nyz, NL, twx, mode, s, done, lpb, gsz);
  VIE_PASS_X3_SIZES(VIE_X)
#undef VIE_X
  return VIE_OK;
}

// Mx = L1 x L2 factorisations with a four-step register x pass.
#define VIE_PASS_X4_SIZES(X) \
  X(40, 30) X(24, 25) X(24, 30) X(30, 30) X(45, 25) X(45, 30) X(50, 30) X(40, 40) X(20, 20)
// (L1, L2, NX) with the line length compiled in: 600 values (12 um at 20 nm
// along x; the ring resonator's 600 y-voxels) into 1200 = 40 x 30.
#define VIE_PASS_X4_FIXED(X) X(40, 30, 600)

template <typename V, int L1, int L2, int LPB, int NX>
static vie_status launch_x4_lpb(bool forward, const PassPtrs<V>& pp, int count, int nx, int nyz, int NL,
                                const V* twx, int mode, cudaStream_t s, bool* done, int gsz) {
  {
    constexpr int R = pitch_mod16(L1 * LPB, LPB);
    constexpr int NT = LPB * (L1 > L2 ? L1 : L2);
    const int P = pitch_mod16(nx, LPB);
    const bool operands = !forward && mode != MODE_PLAIN;   // epilogue rows of x and M
    const size_t smem = (size_t)(L1 * L2 + L1 + L2 + L2 * R + LPB * P + (operands ? 2 * LPB * nx : 0)) * sizeof(V);
    if (smem > 200 * 1024) { *done = false; return VIE_OK; }
    const dim3 blocks((unsigned)((NL + LPB - 1) / LPB), (unsigned)count);
    if (forward) {
      VIE_CUDA_TRY(cudaFuncSetAttribute(pass_a4_kernel<V, L1, L2, LPB, NX>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      VIE_CUDA_TRY(launch_pdl(pass_a4_kernel<V, L1, L2, LPB, NX>, blocks, dim3(NT), smem, s, pp, nx, NL, twx, gsz));
    } else {
      VIE_CUDA_TRY(cudaFuncSetAttribute(pass_c4_kernel<V, L1, L2, LPB, NX>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      VIE_CUDA_TRY(
          launch_pdl(pass_c4_kernel<V, L1, L2, LPB, NX>, blocks, dim3(NT), smem, s, pp, nx, nyz, NL, twx, mode, gsz));
    }
    VIE_LAUNCH_CHECK();
    *done = true;
    return VIE_OK;
  }
}

// Four lines per block, or two when four would leave fewer than one block
// per SM (more blocks hide the latency of the small per-line work), unless
// the plan's tuner chose (lpb = 2 or 4).  Inverse passes with at least four
// blocks of eight lines per SM (complex64) take eight lines when they fit:
// each transposed row read is then 64 contiguous bytes, which matters once
// the workspace no longer fits in L2 (forward passes measured slower so).
template <typename V, int L1, int L2, int NX = 0>
static vie_status launch_x4(bool forward, const PassPtrs<V>& pp, int count, int nx, int nyz, int NL,
                            const V* twx, int mode, cudaStream_t s, bool* done, int lpb, int gsz) {
  if constexpr (sizeof(V) == sizeof(float2) || (L1 <= 30 && L2 <= 30)) {
    if constexpr (sizeof(V) == sizeof(float2)) {
      const long blocks8 = (long)((NL + 7) / 8) * count;
      if (lpb == 8 || (lpb == 0 && !forward && blocks8 >= 4L * kSMs)) {
        vie_status st = launch_x4_lpb<V, L1, L2, 8, NX>(forward, pp, count, nx, nyz, NL, twx, mode, s, done, gsz);
        if (st != VIE_OK || *done) return st;
      }
    }
    if constexpr (sizeof(V) == sizeof(float2) && NX > 0) {
      if (lpb == 5 || (lpb == 0 && x_lines_five(NL, count)))
        return launch_x4_lpb<V, L1, L2, 5, NX>(forward, pp, count, nx, nyz, NL, twx, mode, s, done, gsz);
    }
    const long blocks4 = (long)((NL + 3) / 4) * count;
    if (lpb == 2) return launch_x4_lpb<V, L1, L2, 2, NX>(forward, pp, count, nx, nyz, NL, twx, mode, s, done, gsz);
    if (lpb == 4) return launch_x4_lpb<V, L1, L2, 4, NX>(forward, pp, count, nx, nyz, NL, twx, mode, s, done, gsz);
    if (blocks4 < kSMs)
      return launch_x4_lpb<V, L1, L2, 2, NX>(forward, pp, count, nx, nyz, NL, twx, mode, s, done, gsz);
    return launch_x4_lpb<V, L1, L2, 4, NX>(forward, pp, count, nx, nyz, NL, twx, mode, s, done, gsz);
  } else {
    *done = false;
    return VIE_OK;
  }
}

// factor (L1, L2) of Mx with a compiled four-step kernel, or (0, 0)
void x4_factors(int mx, int* l1, int* l2) {
  *l1 = 0;
  *l2 = 0;
#define VIE_X(a, b) if (mx == a * b && *l1 == 0) { *l1 = a; *l2 = b; }
  VIE_PASS_X4_SIZES(VIE_X)
#undef VIE_X
}

template <typename V>
static vie_status dispatch_x4(bool forward, int l1, int l2, const PassPtrs<V>& pp, int count, int nx, int nyz,
                              int NL, const V* twx, int mode, cudaStream_t s, bool* done, int lpb, int gsz) {
  *done = false;
#define VIE_X(a, b) \
  if (l1 == a && l2 == b) return launch_x4<V, a, b>(forward, pp, count, nx, nyz, NL, twx, mode, s, done, lpb, gsz);
#define VIE_Y(a, b, c)                      \
  if (l1 == a && l2 == b && nx == c)          \
    return launch_x4<V, a, b, c>(forward, pp, count, nx, nyz, NL, twx, mode, s, done, lpb, gsz);
  VIE_PASS_X4_FIXED(VIE_Y)
#undef VIE_Y
  VIE_PASS_X4_SIZES(VIE_X)
#undef VIE_X
  return VIE_OK;
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
// Planes that neither the register pass B nor the one-CTA generic pass B can
// hold take the split pass B when a z-stage kernel exists for Mz.
static bool pass_b_needs_more_than_one_cta(int My, int Mz, size_t vbytes) {
  return (size_t)(My + Mz + 2 * 3 * Mz * (My + 1)) * vbytes > 220 * 1024;
}

size_t pass_b_split_elems(int ny, int nz, int Mx, int My, int Mz) {
  (void)ny;
  if (!pass_b_needs_more_than_one_cta(My, Mz, sizeof(double2)) || !pass_bz_available(Mz)) return 0;
  return (size_t)Mx * My * 3 * nz;
}

// Generic (shared-memory Stockham) x-pass kernels for `n`-value lines
// transformed at length rd.len: pass_a_kernel forward, pass_c_kernel inverse.
template <typename V>
static vie_status launch_x_generic(bool forward, const PassPtrs<V>& pp, int count, int n, int nyz, int NL,
                                   const Radices& rd, const V* tw, int mode, cudaStream_t s, int gsz) {
  const size_t line_bytes = (size_t)2 * (rd.len + 1) * sizeof(V);
  const size_t tw_bytes = (size_t)rd.len * sizeof(V);
  int lpb = 4;
  while (lpb > 1 && tw_bytes + lpb * line_bytes > 200 * 1024) lpb >>= 1;
  const size_t smem = tw_bytes + lpb * line_bytes;
  if (smem > 220 * 1024) {
    set_error("FFT length %d too large for the line-pass shared memory", rd.len);
    return VIE_ERR_INVALID;
  }
  const dim3 blocks((unsigned)((NL + lpb - 1) / lpb), (unsigned)count);
  if (forward) {
    VIE_CUDA_TRY(cudaFuncSetAttribute(pass_a_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    pass_a_kernel<V><<<blocks, 256, smem, s>>>(pp, n, NL, rd, tw, lpb, gsz);
  } else {
    VIE_CUDA_TRY(cudaFuncSetAttribute(pass_c_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    pass_c_kernel<V><<<blocks, 256, smem, s>>>(pp, n, nyz, NL, rd, tw, lpb, mode, gsz);
  }
  VIE_LAUNCH_CHECK();
  return VIE_OK;
}

// Split pass B (B1, B2, B3 above) on the workspaces pp.work / pp.work2.
template <typename V>
static vie_status run_split_b(const vie_plan* p, const PassPtrs<V>& pp, int count, const PassBGeom& g,
                              const V* twy, const V* twz, cudaStream_t s) {
  const int NLy = g.Mx * 3 * g.nz;
  int l1 = 0, l2 = 0;
  x4_factors(g.My, &l1, &l2);
  PassPtrs<V> p1 = pp;   // B1: lines of the slab -> Y
  PassPtrs<V> p3 = pp;   // B3: Y -> lines of the slab
  for (int k = 0; k < count; ++k) {
    p1.x[k] = pp.work[k];
    p1.work[k] = pp.work2[k];
    p3.work[k] = pp.work2[k];
    p3.y[k] = pp.work[k];
  }
  bool done = false;
  vie_status st = VIE_OK;
  const int gsz = 3 * g.nz;   // one group of lines per kx: Y[kx][ky][l]
  if (l1) st = dispatch_x4<V>(true, l1, l2, p1, count, g.ny, 1, NLy, twy, MODE_PLAIN, s, &done, 0, gsz);
  if (st == VIE_OK && !done)
    st = launch_x_generic<V>(true, p1, count, g.ny, 1, NLy, radices_of(p->ax[1]), twy, MODE_PLAIN, s, gsz);
  if (st == VIE_OK) st = dispatch_pass_bz<V>(pp, count, g, twz, s);
  done = false;
  if (st == VIE_OK && l1)
    st = dispatch_x4<V>(false, l1, l2, p3, count, g.ny, 1, NLy, twy, MODE_PLAIN, s, &done, 0, gsz);
  if (st == VIE_OK && !done)
    st = launch_x_generic<V>(false, p3, count, g.ny, 1, NLy, radices_of(p->ax[1]), twy, MODE_PLAIN, s, gsz);
  return st;
}

// The three passes for `count` problems of one shape (count <= kMaxBatch).
template <typename V>
static vie_status run_passes(const vie_plan* p, const PassPtrs<V>& pp, int count, const V* twx, const V* twy,
                             const V* twz, int mode, cudaStream_t s) {
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  const int Mx = p->m[0], My = p->m[1], Mz = p->m[2];
  const int NL = 3 * ny * nz;
  const int threads = 256;
  // generic x passes: lines per block from the shared-memory budget
  const size_t line_bytes = (size_t)2 * (Mx + 1) * sizeof(V);
  const size_t tw_bytes = (size_t)Mx * sizeof(V);
  int lpb = 4;
  while (lpb > 1 && tw_bytes + lpb * line_bytes > 200 * 1024) lpb >>= 1;
  const size_t smem_ac = tw_bytes + lpb * line_bytes;
  if (smem_ac > 220 * 1024) {
    set_error("Mx = %d too large for the x-pass shared memory", Mx);
    return VIE_ERR_INVALID;
  }
  const size_t smem_b = (size_t)(My + Mz + 2 * 3 * Mz * (My + 1)) * sizeof(V);
  const dim3 blocks_ac((unsigned)((NL + lpb - 1) / lpb), (unsigned)count);
  int l1 = 0, l2 = 0, a1 = 0, a2 = 0, a3 = 0;
  x4_factors(Mx, &l1, &l2);
  x3_factors(Mx, &a1, &a2, &a3);
  bool done = false;
  vie_status st = VIE_OK;
  // x passes: three-factor kernels (x_lpb < 0: -x_lpb lines per block; 0:
  // the default for the forward pass where they exist), else four-step
  // (x_lpb > 0), else generic
  if (a1 && p->x_lpb <= 0) {
    st = dispatch_x3<V>(true, a1, a2, a3, pp, count, nx, ny * nz, NL, twx, mode, s, &done,
                        p->x_lpb < 0 ? -p->x_lpb : 0, NL);
    if (st != VIE_OK) return st;
  }
  if (!done && l1) {
    st = dispatch_x4<V>(true, l1, l2, pp, count, nx, ny * nz, NL, twx, mode, s, &done, p->x_lpb > 0 ? p->x_lpb : 0,
                        NL);
    if (st != VIE_OK) return st;
  }
  if (!done) {
    VIE_CUDA_TRY(cudaFuncSetAttribute(pass_a_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_ac));
    pass_a_kernel<V><<<blocks_ac, threads, smem_ac, s>>>(pp, nx, NL, radices_of(p->ax[0]), twx, lpb, NL);
    VIE_LAUNCH_CHECK();
  }
  PassBGeom g{ny, nz, NL, Mx, My, Mz, p->kf[1], p->kf[2]};
  st = dispatch_pass_b_reg<V>(pp, count, g, twy, twz, s, &done);
  if (st != VIE_OK) return st;
  if (!done && smem_b > 220 * 1024 && pp.work2[0] && pass_bz_available(Mz)) {
    st = run_split_b<V>(p, pp, count, g, twy, twz, s);
    if (st != VIE_OK) return st;
    done = true;
  }
  if (!done && smem_b > 220 * 1024) {
    st = launch_pass_b_cluster<V>(pp, count, g, radices_of(p->ax[1]), radices_of(p->ax[2]), twy, twz, s);
    if (st != VIE_OK) return st;
    done = true;
  }
  if (!done) {
    VIE_CUDA_TRY(cudaFuncSetAttribute(pass_b_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
    pass_b_kernel<V><<<dim3((unsigned)Mx, (unsigned)count), threads, smem_b, s>>>(pp, g, radices_of(p->ax[1]),
                                                                                radices_of(p->ax[2]), twy, twz);
    VIE_LAUNCH_CHECK();
  }
  done = false;
  // inverse: three-factor only when chosen (x_lpb_inv < 0) or when no
  // four-step kernel exists for Mx; the four-step inverse, whose blocks read
  // 32-byte rows of the transposed workspace, measured faster on the guide
  if (a1 && (p->x_lpb_inv < 0 || (p->x_lpb_inv == 0 && !l1))) {
    st = dispatch_x3<V>(false, a1, a2, a3, pp, count, nx, ny * nz, NL, twx, mode, s, &done,
                        p->x_lpb_inv < 0 ? -p->x_lpb_inv : 0, NL);
    if (st != VIE_OK) return st;
  }
  if (!done && l1) {
    st = dispatch_x4<V>(false, l1, l2, pp, count, nx, ny * nz, NL, twx, mode, s, &done,
                        p->x_lpb_inv > 0 ? p->x_lpb_inv : 0, NL);
    if (st != VIE_OK) return st;
  }
  if (!done) {
    VIE_CUDA_TRY(cudaFuncSetAttribute(pass_c_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_ac));
    pass_c_kernel<V><<<blocks_ac, threads, smem_ac, s>>>(pp, nx, ny * nz, NL, radices_of(p->ax[0]), twx, lpb, mode,
                                                        NL);
    VIE_LAUNCH_CHECK();
  }
  return VIE_OK;
}

// ---------------------------------------------------------------------------
// JM-VIE (Sec. 3): the operator on six components (u_e, u_m) per voxel,
//   v_e = T * u_e - j kappa C x u_m,   v_m = T * u_m + j kappa C x u_e,
// y = u - M v (M_eps on the electric, M_mu on the magnetic components), or
// y = M (v - u) for a right-hand side.  The x passes are those of the J-VIE
// on 6 ny nz lines; pass B transforms the six components of one kx plane
// and applies the symmetric 3 x 3 spectrum of T to each current and the
// cross product with the three curl spectra C_a (C_a odd along axis a:
// folding along a flips its sign) between them.
// ---------------------------------------------------------------------------
template <typename V>
__global__ void __launch_bounds__(256) pass_b_jm_kernel(V* __restrict__ work, const V* __restrict__ ghat,
                                                        const V* __restrict__ chat, PassBGeom g, Radices ry,
                                                        Radices rz, const V* __restrict__ twyg,
                                                        const V* __restrict__ twzg, double kappa) {
  typedef typename real_of<V>::type R;
  pdl_wait();
  extern __shared__ unsigned char smem_raw[];
  const int kx = blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int ny = g.ny, nz = g.nz, My = g.My, Mz = g.Mz;
  const int pz = Mz + 1, py = My + 1;
  const int buf = 6 * Mz * py;   // >= 6 * ny * pz since My >= ny
  V* twy = reinterpret_cast<V*>(smem_raw);
  V* twz = twy + My;
  V* U = twz + Mz;
  V* W = U + buf;
  for (int i = tid; i < My; i += nth) twy[i] = twyg[i];
  for (int i = tid; i < Mz; i += nth) twz[i] = twzg[i];
  V* slab = work + (size_t)kx * g.NL;
  for (int e = tid; e < 6 * ny * Mz; e += nth) {
    const int row = e / Mz, z = e - row * Mz;   // row = c*ny + y
    const int c = row / ny, y = row - c * ny;
    U[row * pz + z] = (z < nz) ? slab[(c * nz + z) * ny + y] : zero_c<V>();
  }
  __syncthreads();
  V* zr = fft_lines<V, false>(U, W, rz, pz, 6 * ny, twz, tid, nth);
  V* other = (zr == U) ? W : U;
  for (int e = tid; e < 6 * Mz * My; e += nth) {
    const int row = e / My, y = e - row * My;   // row = c*Mz + kz
    const int c = row / Mz, kz = row - c * Mz;
    other[row * py + y] = (y < ny) ? zr[(c * ny + y) * pz + kz] : zero_c<V>();
  }
  __syncthreads();
  V* yr = fft_lines<V, false>(other, zr, ry, py, 6 * Mz, twy, tid, nth);
  {
    const bool fx = kx > g.Mx - kx;
    const int kxf = fx ? g.Mx - kx : kx;
    const size_t cs = (size_t)g.Kz * g.Ky;
    const V* G = ghat + (size_t)kxf * 6 * cs;
    const V* Cc = chat + (size_t)kxf * 3 * cs;
    const R kap = (R)kappa;
    for (int e = tid; e < Mz * My; e += nth) {
      const int kz = e / My, ky = e - kz * My;
      const bool fy = ky > My - ky, fz = kz > Mz - kz;
      const int kyf = fy ? My - ky : ky, kzf = fz ? Mz - kz : kz;
      const size_t o = (size_t)kzf * g.Ky + kyf;
      V gxx = G[o], gyy = G[cs + o], gzz = G[2 * cs + o];
      V gxy = G[3 * cs + o], gxz = G[4 * cs + o], gyz = G[5 * cs + o];
      if (fx ^ fy) gxy = scale(gxy, (R)-1);
      if (fx ^ fz) gxz = scale(gxz, (R)-1);
      if (fy ^ fz) gyz = scale(gyz, (R)-1);
      // j kappa C_a, with the fold signs
      V cx = Cc[o], cy = Cc[cs + o], cz = Cc[2 * cs + o];
      if (fx) cx = scale(cx, (R)-1);
      if (fy) cy = scale(cy, (R)-1);
      if (fz) cz = scale(cz, (R)-1);
      cx = scale(mul_pi(cx), kap);
      cy = scale(mul_pi(cy), kap);
      cz = scale(mul_pi(cz), kap);
      V* p[6];
      V u[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        p[c] = yr + (c * Mz + kz) * py + ky;
        u[c] = *p[c];
      }
      // T u for each current
      const V te0 = add(add(mul(gxx, u[0]), mul(gxy, u[1])), mul(gxz, u[2]));
      const V te1 = add(add(mul(gxy, u[0]), mul(gyy, u[1])), mul(gyz, u[2]));
      const V te2 = add(add(mul(gxz, u[0]), mul(gyz, u[1])), mul(gzz, u[2]));
      const V tm0 = add(add(mul(gxx, u[3]), mul(gxy, u[4])), mul(gxz, u[5]));
      const V tm1 = add(add(mul(gxy, u[3]), mul(gyy, u[4])), mul(gyz, u[5]));
      const V tm2 = add(add(mul(gxz, u[3]), mul(gyz, u[4])), mul(gzz, u[5]));
      // (j kappa C) x u_m and (j kappa C) x u_e
      const V xm0 = sub(mul(cy, u[5]), mul(cz, u[4]));
      const V xm1 = sub(mul(cz, u[3]), mul(cx, u[5]));
      const V xm2 = sub(mul(cx, u[4]), mul(cy, u[3]));
      const V xe0 = sub(mul(cy, u[2]), mul(cz, u[1]));
      const V xe1 = sub(mul(cz, u[0]), mul(cx, u[2]));
      const V xe2 = sub(mul(cx, u[1]), mul(cy, u[0]));
      *p[0] = sub(te0, xm0);
      *p[1] = sub(te1, xm1);
      *p[2] = sub(te2, xm2);
      *p[3] = add(tm0, xe0);
      *p[4] = add(tm1, xe1);
      *p[5] = add(tm2, xe2);
    }
  }
  __syncthreads();
  V* spare = (yr == U) ? W : U;
  V* yi = fft_lines<V, true>(yr, spare, ry, py, 6 * Mz, twy, tid, nth);
  V* other2 = (yi == U) ? W : U;
  for (int e = tid; e < 6 * ny * Mz; e += nth) {
    const int row = e / Mz, kz = e - row * Mz;
    const int c = row / ny, y = row - c * ny;
    other2[row * pz + kz] = yi[(c * Mz + kz) * py + y];
  }
  __syncthreads();
  V* spare2 = (other2 == U) ? W : U;
  V* zi = fft_lines<V, true>(other2, spare2, rz, pz, 6 * ny, twz, tid, nth);
  for (int e = tid; e < g.NL; e += nth) {
    const int y = e % ny, cz = e / ny;
    const int z = cz % nz, c = cz / nz;
    slab[e] = zi[(c * ny + y) * pz + z];
  }
}

// The JM-VIE pass B with register FFTs (as pass_b_reg_kernel, six
// components): one CTA per kx, z and y lines of the six components in
// registers, the N spectrum and the curl spectra of this kx staged in shared
// memory while the forward transforms run.
template <typename V, int MY, int MZ, int NY, int NZ>
__global__ void __launch_bounds__(256) pass_b_reg_jm_kernel(V* __restrict__ work, const V* __restrict__ ghat,
                                                            const V* __restrict__ chat, PassBGeom g,
                                                            const V* __restrict__ twyg, const V* __restrict__ twzg,
                                                            double kappa) {
  typedef typename real_of<V>::type R;
  constexpr int PY = (MY % 2 == 0) ? MY + 1 : MY;
  constexpr int PZ = (MZ % 2 == 0) ? MZ + 1 : MZ;
  extern __shared__ unsigned char smem_raw[];
  V* twy = reinterpret_cast<V*>(smem_raw);
  V* twz = twy + MY;
  V* S1 = twz + MZ;
  V* S2 = S1 + 6 * MZ * PY;
  V* Gs = S2 + 6 * g.ny * PZ;          // N spectrum chunk (6 Kz Ky), then the curl chunk (3 Kz Ky)
  const int kx = blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int ny = NY > 0 ? NY : g.ny, nz = NZ > 0 ? NZ : g.nz;
  const bool fx = kx > g.Mx - kx;
  const int kxf = fx ? g.Mx - kx : kx;
  const int cs = g.Kz * g.Ky;
  pdl_launch_dependents();
  for (int i = tid; i < MY; i += nth) __pipeline_memcpy_async(twy + i, twyg + i, sizeof(V));
  for (int i = tid; i < MZ; i += nth) __pipeline_memcpy_async(twz + i, twzg + i, sizeof(V));
  __pipeline_commit();
  {
    const V* G = ghat + (size_t)kxf * 6 * cs;
    const V* C = chat + (size_t)kxf * 3 * cs;
    for (int i = tid; i < 6 * cs; i += nth) __pipeline_memcpy_async(Gs + i, G + i, sizeof(V));
    for (int i = tid; i < 3 * cs; i += nth) __pipeline_memcpy_async(Gs + 6 * cs + i, C + i, sizeof(V));
    __pipeline_commit();
  }
  pdl_wait();
  __pipeline_wait_prior(1);
  __syncthreads();
  V* slab = work + (size_t)kx * g.NL;
  for (int line = tid; line < 6 * ny; line += nth) {
    const int c = line / ny, y = line - c * ny;
    V a[MZ];
#pragma unroll
    for (int z = 0; z < MZ; ++z) a[z] = (z < nz) ? slab[(c * nz + z) * ny + y] : zero_c<V>();
    reg_fft<V, false, MZ>(a, twz);
#pragma unroll
    for (int kz = 0; kz < MZ; ++kz) S1[(c * MZ + kz) * PY + y] = a[kz];
  }
  __syncthreads();
  for (int line = tid; line < 6 * MZ; line += nth) {
    V a[MY];
#pragma unroll
    for (int y = 0; y < MY; ++y) a[y] = (y < ny) ? S1[line * PY + y] : zero_c<V>();
    reg_fft<V, false, MY>(a, twy);
#pragma unroll
    for (int ky = 0; ky < MY; ++ky) S1[line * PY + ky] = a[ky];
  }
  __pipeline_wait_prior(0);
  __syncthreads();
  {
    const V* G = Gs;
    const V* Cc = Gs + 6 * cs;
    const R kap = (R)kappa;
    for (int e = tid; e < MZ * MY; e += nth) {
      const int kz = e / MY, ky = e - kz * MY;
      const bool fy = ky > MY - ky, fz = kz > MZ - kz;
      const int kyf = fy ? MY - ky : ky, kzf = fz ? MZ - kz : kz;
      const int o = kzf * g.Ky + kyf;
      V gxx = G[o], gyy = G[cs + o], gzz = G[2 * cs + o];
      V gxy = G[3 * cs + o], gxz = G[4 * cs + o], gyz = G[5 * cs + o];
      if (fx ^ fy) gxy = scale(gxy, (R)-1);
      if (fx ^ fz) gxz = scale(gxz, (R)-1);
      if (fy ^ fz) gyz = scale(gyz, (R)-1);
      V cx = Cc[o], cy = Cc[cs + o], cz = Cc[2 * cs + o];
      if (fx) cx = scale(cx, (R)-1);
      if (fy) cy = scale(cy, (R)-1);
      if (fz) cz = scale(cz, (R)-1);
      cx = scale(mul_pi(cx), kap);
      cy = scale(mul_pi(cy), kap);
      cz = scale(mul_pi(cz), kap);
      V u[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) u[c] = S1[(c * MZ + kz) * PY + ky];
      const V te0 = add(add(mul(gxx, u[0]), mul(gxy, u[1])), mul(gxz, u[2]));
      const V te1 = add(add(mul(gxy, u[0]), mul(gyy, u[1])), mul(gyz, u[2]));
      const V te2 = add(add(mul(gxz, u[0]), mul(gyz, u[1])), mul(gzz, u[2]));
      const V tm0 = add(add(mul(gxx, u[3]), mul(gxy, u[4])), mul(gxz, u[5]));
      const V tm1 = add(add(mul(gxy, u[3]), mul(gyy, u[4])), mul(gyz, u[5]));
      const V tm2 = add(add(mul(gxz, u[3]), mul(gyz, u[4])), mul(gzz, u[5]));
      S1[(0 * MZ + kz) * PY + ky] = sub(te0, sub(mul(cy, u[5]), mul(cz, u[4])));
      S1[(1 * MZ + kz) * PY + ky] = sub(te1, sub(mul(cz, u[3]), mul(cx, u[5])));
      S1[(2 * MZ + kz) * PY + ky] = sub(te2, sub(mul(cx, u[4]), mul(cy, u[3])));
      S1[(3 * MZ + kz) * PY + ky] = add(tm0, sub(mul(cy, u[2]), mul(cz, u[1])));
      S1[(4 * MZ + kz) * PY + ky] = add(tm1, sub(mul(cz, u[0]), mul(cx, u[2])));
      S1[(5 * MZ + kz) * PY + ky] = add(tm2, sub(mul(cx, u[1]), mul(cy, u[0])));
    }
  }
  __syncthreads();
  for (int line = tid; line < 6 * MZ; line += nth) {
    const int c = line / MZ, kz = line - c * MZ;
    V a[MY];
#pragma unroll
    for (int ky = 0; ky < MY; ++ky) a[ky] = S1[line * PY + ky];
    reg_fft<V, true, MY>(a, twy);
#pragma unroll
    for (int y = 0; y < MY; ++y)
      if (y < ny) S2[(c * ny + y) * PZ + kz] = a[y];
  }
  __syncthreads();
  for (int line = tid; line < 6 * ny; line += nth) {
    const int c = line / ny, y = line - c * ny;
    V a[MZ];
#pragma unroll
    for (int kz = 0; kz < MZ; ++kz) a[kz] = S2[line * PZ + kz];
    reg_fft<V, true, MZ>(a, twz);
#pragma unroll
    for (int z = 0; z < MZ; ++z)
      if (z < nz) slab[(c * nz + z) * ny + y] = a[z];
  }
}

template <typename V, int MY, int MZ, int NY, int NZ>
static vie_status try_pass_b_reg_jm(V* work, const V* ghat, const V* chat, const PassBGeom& g, const V* twy,
                                    const V* twz, double kappa, cudaStream_t s, bool* done) {
  *done = false;
  // complex128 lines of these lengths would spill registers (the six-current
  // multiply holds 12 spectra): those keep the generic JM pass
  if constexpr (sizeof(V) == sizeof(float2)) {
    constexpr int PY = (MY % 2 == 0) ? MY + 1 : MY;
    constexpr int PZ = (MZ % 2 == 0) ? MZ + 1 : MZ;
    const size_t smem = (size_t)(MY + MZ + 6 * MZ * PY + 6 * g.ny * PZ + 9 * g.Kz * g.Ky) * sizeof(V);
    if (smem > 220 * 1024) return VIE_OK;
    VIE_CUDA_TRY(cudaFuncSetAttribute(pass_b_reg_jm_kernel<V, MY, MZ, NY, NZ>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int lines = 6 * (g.ny > MZ ? g.ny : MZ);
    int threads = ((lines + 31) / 32) * 32;
    if (threads > 256) threads = 256;
    VIE_CUDA_TRY(launch_pdl(pass_b_reg_jm_kernel<V, MY, MZ, NY, NZ>, dim3((unsigned)g.Mx), dim3(threads), smem, s,
                            work, ghat, chat, g, twy, twz, kappa));
    *done = true;
  }
  return VIE_OK;
}

// register JM pass B for the compiled cross-sections (the guide's 23 x 11
// with My 45 or 48 and Mz 24)
template <typename V>
static vie_status dispatch_pass_b_reg_jm(V* work, const V* ghat, const V* chat, const PassBGeom& g, const V* twy,
                                         const V* twz, double kappa, cudaStream_t s, bool* done) {
  *done = false;
#define VIE_Y(a, b, c, d)                                  \
  if (g.My == a && g.Mz == b && g.ny == c && g.nz == d)     \
    return try_pass_b_reg_jm<V, a, b, c, d>(work, ghat, chat, g, twy, twz, kappa, s, done);
  VIE_PASS_B_REG_FIXED(VIE_Y)
#undef VIE_Y
  return VIE_OK;
}

// One line of `len` values at a[0], a[stride], ...: gathered into the warp's
// scratch pair (sa, sb), transformed with Stockham stages by the 32 lanes of
// the warp (warp-synchronous), scattered back.  Every lane of the warp calls
// it with the same arguments.
template <typename V, bool INV>
__device__ void fft_line_warp(V* a, int stride, V* sa, V* sb, const Radices& rd, const V* tw, int lane) {
  for (int i = lane; i < rd.len; i += 32) sa[i] = a[(size_t)i * stride];
  __syncwarp();
  V* src = sa;
  V* dst = sb;
  int s = 1;
  for (int st = 0; st < rd.nstages; ++st) {
    const int r = rd.r[st];
    stockham_stage<V, INV>(src, dst, rd.len, rd.len, 1, r, s, tw, lane, 32);
    __syncwarp();
    V* t = src; src = dst; dst = t;
    s *= r;
  }
  for (int i = lane; i < rd.len; i += 32) a[(size_t)i * stride] = src[i];
  __syncwarp();
}

// The JM-VIE pass B for planes too large for two plane buffers in shared
// memory: one plane buffer P[(c Mz + kz) (My + 1) + ky] and, per warp, a
// scratch pair of the longer line length; each line is transformed by one
// warp.  z lines (stride My + 1) only for y < ny and, on the way back, only
// the z < nz outputs are written to the slab.
template <typename V>
__global__ void __launch_bounds__(256) pass_b_jm_lines_kernel(V* __restrict__ work, const V* __restrict__ ghat,
                                                              const V* __restrict__ chat, PassBGeom g, Radices ry,
                                                              Radices rz, const V* __restrict__ twyg,
                                                              const V* __restrict__ twzg, double kappa) {
  typedef typename real_of<V>::type R;
  pdl_wait();
  extern __shared__ unsigned char smem_raw[];
  const int kx = blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nth >> 5;
  const int ny = g.ny, nz = g.nz, My = g.My, Mz = g.Mz;
  const int py = My + 1;
  const int lmax = My > Mz ? My : Mz;
  V* twy = reinterpret_cast<V*>(smem_raw);
  V* twz = twy + My;
  V* P = twz + Mz;
  V* scr = P + 6 * Mz * py + warp * 2 * lmax;
  for (int i = tid; i < My; i += nth) twy[i] = twyg[i];
  for (int i = tid; i < Mz; i += nth) twz[i] = twzg[i];
  V* slab = work + (size_t)kx * g.NL;
  for (int e = tid; e < 6 * Mz * py; e += nth) {
    const int row = e / py, y = e - row * py;   // row = c*Mz + z
    const int c = row / Mz, z = row - c * Mz;
    P[e] = (z < nz && y < ny) ? slab[(c * nz + z) * ny + y] : zero_c<V>();
  }
  __syncthreads();
  for (int line = warp; line < 6 * ny; line += nwarps) {
    const int c = line / ny, y = line - c * ny;
    fft_line_warp<V, false>(P + (size_t)c * Mz * py + y, py, scr, scr + lmax, rz, twz, lane);
  }
  __syncthreads();
  for (int line = warp; line < 6 * Mz; line += nwarps)
    fft_line_warp<V, false>(P + (size_t)line * py, 1, scr, scr + lmax, ry, twy, lane);
  __syncthreads();
  {
    const bool fx = kx > g.Mx - kx;
    const int kxf = fx ? g.Mx - kx : kx;
    const size_t cs = (size_t)g.Kz * g.Ky;
    const V* G = ghat + (size_t)kxf * 6 * cs;
    const V* Cc = chat + (size_t)kxf * 3 * cs;
    const R kap = (R)kappa;
    for (int e = tid; e < Mz * My; e += nth) {
      const int kz = e / My, ky = e - kz * My;
      const bool fy = ky > My - ky, fz = kz > Mz - kz;
      const int kyf = fy ? My - ky : ky, kzf = fz ? Mz - kz : kz;
      const size_t o = (size_t)kzf * g.Ky + kyf;
      V gxx = G[o], gyy = G[cs + o], gzz = G[2 * cs + o];
      V gxy = G[3 * cs + o], gxz = G[4 * cs + o], gyz = G[5 * cs + o];
      if (fx ^ fy) gxy = scale(gxy, (R)-1);
      if (fx ^ fz) gxz = scale(gxz, (R)-1);
      if (fy ^ fz) gyz = scale(gyz, (R)-1);
      V cx = Cc[o], cy = Cc[cs + o], cz = Cc[2 * cs + o];
      if (fx) cx = scale(cx, (R)-1);
      if (fy) cy = scale(cy, (R)-1);
      if (fz) cz = scale(cz, (R)-1);
      cx = scale(mul_pi(cx), kap);
      cy = scale(mul_pi(cy), kap);
      cz = scale(mul_pi(cz), kap);
      V* q[6];
      V u[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        q[c] = P + (c * Mz + kz) * py + ky;
        u[c] = *q[c];
      }
      const V te0 = add(add(mul(gxx, u[0]), mul(gxy, u[1])), mul(gxz, u[2]));
      const V te1 = add(add(mul(gxy, u[0]), mul(gyy, u[1])), mul(gyz, u[2]));
      const V te2 = add(add(mul(gxz, u[0]), mul(gyz, u[1])), mul(gzz, u[2]));
      const V tm0 = add(add(mul(gxx, u[3]), mul(gxy, u[4])), mul(gxz, u[5]));
      const V tm1 = add(add(mul(gxy, u[3]), mul(gyy, u[4])), mul(gyz, u[5]));
      const V tm2 = add(add(mul(gxz, u[3]), mul(gyz, u[4])), mul(gzz, u[5]));
      *q[0] = sub(te0, sub(mul(cy, u[5]), mul(cz, u[4])));
      *q[1] = sub(te1, sub(mul(cz, u[3]), mul(cx, u[5])));
      *q[2] = sub(te2, sub(mul(cx, u[4]), mul(cy, u[3])));
      *q[3] = add(tm0, sub(mul(cy, u[2]), mul(cz, u[1])));
      *q[4] = add(tm1, sub(mul(cz, u[0]), mul(cx, u[2])));
      *q[5] = add(tm2, sub(mul(cx, u[1]), mul(cy, u[0])));
    }
  }
  __syncthreads();
  for (int line = warp; line < 6 * Mz; line += nwarps)
    fft_line_warp<V, true>(P + (size_t)line * py, 1, scr, scr + lmax, ry, twy, lane);
  __syncthreads();
  for (int line = warp; line < 6 * ny; line += nwarps) {
    const int c = line / ny, y = line - c * ny;
    fft_line_warp<V, true>(P + (size_t)c * Mz * py + y, py, scr, scr + lmax, rz, twz, lane);
  }
  __syncthreads();
  for (int e = tid; e < g.NL; e += nth) {
    const int y = e % ny, cz = e / ny;
    const int z = cz % nz, c = cz / nz;
    slab[e] = P[(c * Mz + z) * py + y];
  }
}

size_t jm_pass_b_lines_smem(int My, int Mz, size_t vbytes) {
  const int lmax = My > Mz ? My : Mz;
  return (size_t)(My + Mz + 6 * Mz * (My + 1) + 8 * 2 * lmax) * vbytes;
}

size_t jm_pass_b_smem(int My, int Mz, size_t vbytes) {
  return (size_t)(My + Mz + 2 * 6 * Mz * (My + 1)) * vbytes;
}

template <typename V>
static vie_status run_jm(vie_plan* p, const V* x, V* y, const V* ghat, const V* chat, const V* Mc, const V* twx,
                         const V* twy, const V* twz, int mode, cudaStream_t s) {
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  const int Mx = p->m[0], My = p->m[1], Mz = p->m[2];
  const int NL = 6 * ny * nz;
  const size_t smem_b = jm_pass_b_smem(My, Mz, sizeof(V));
  const size_t smem_bl = jm_pass_b_lines_smem(My, Mz, sizeof(V));
  if (smem_bl > 220 * 1024) {
    set_error("the JM-VIE operator needs the 6 x %d x %d plane of one kx in one CTA's shared memory", My, Mz);
    return VIE_ERR_INVALID;
  }
  PassPtrs<V> pp;
  memset(&pp, 0, sizeof(pp));
  pp.x[0] = x;
  pp.y[0] = y;
  pp.work[0] = (V*)p->jm_work;
  pp.ghat[0] = ghat;
  pp.M[0] = Mc;
  const size_t line_bytes = (size_t)2 * (Mx + 1) * sizeof(V);
  const size_t tw_bytes = (size_t)Mx * sizeof(V);
  int lpb = 4;
  while (lpb > 1 && tw_bytes + lpb * line_bytes > 200 * 1024) lpb >>= 1;
  const size_t smem_ac = tw_bytes + lpb * line_bytes;
  if (smem_ac > 220 * 1024) {
    set_error("Mx = %d too large for the x-pass shared memory", Mx);
    return VIE_ERR_INVALID;
  }
  const dim3 blocks_ac((unsigned)((NL + lpb - 1) / lpb), 1);
  int l1 = 0, l2 = 0, a1 = 0, a2 = 0, a3 = 0;
  x4_factors(Mx, &l1, &l2);
  x3_factors(Mx, &a1, &a2, &a3);
  bool done = false;
  vie_status st = VIE_OK;
  if (a1) {
    st = dispatch_x3<V>(true, a1, a2, a3, pp, 1, nx, NL, NL, twx, mode, s, &done, 0, NL);
    if (st != VIE_OK) return st;
  }
  if (!done && l1) {
    st = dispatch_x4<V>(true, l1, l2, pp, 1, nx, NL, NL, twx, mode, s, &done, 0, NL);
    if (st != VIE_OK) return st;
  }
  if (!done) {
    VIE_CUDA_TRY(cudaFuncSetAttribute(pass_a_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_ac));
    pass_a_kernel<V><<<blocks_ac, 256, smem_ac, s>>>(pp, nx, NL, radices_of(p->ax[0]), twx, lpb, NL);
    VIE_LAUNCH_CHECK();
  }
  PassBGeom g{ny, nz, NL, Mx, My, Mz, p->kf[1], p->kf[2]};
  st = dispatch_pass_b_reg_jm<V>((V*)p->jm_work, ghat, chat, g, twy, twz, p->kappa, s, &done);
  if (st != VIE_OK) return st;
  if (!done && smem_b <= 220 * 1024) {
    VIE_CUDA_TRY(cudaFuncSetAttribute(pass_b_jm_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
    pass_b_jm_kernel<V><<<(unsigned)Mx, 256, smem_b, s>>>((V*)p->jm_work, ghat, chat, g, radices_of(p->ax[1]),
                                                          radices_of(p->ax[2]), twy, twz, p->kappa);
    VIE_LAUNCH_CHECK();
    done = true;
  }
  if (!done) {
    VIE_CUDA_TRY(cudaFuncSetAttribute(pass_b_jm_lines_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem_bl));
    pass_b_jm_lines_kernel<V><<<(unsigned)Mx, 256, smem_bl, s>>>((V*)p->jm_work, ghat, chat, g,
                                                                 radices_of(p->ax[1]), radices_of(p->ax[2]), twy,
                                                                 twz, p->kappa);
    VIE_LAUNCH_CHECK();
  }
  done = false;
  if (a1) {
    st = dispatch_x3<V>(false, a1, a2, a3, pp, 1, nx, NL, NL, twx, mode, s, &done, 0, NL);
    if (st != VIE_OK) return st;
  }
  if (!done && l1) {
    st = dispatch_x4<V>(false, l1, l2, pp, 1, nx, NL, NL, twx, mode, s, &done, 0, NL);
    if (st != VIE_OK) return st;
  }
  if (!done) {
    VIE_CUDA_TRY(cudaFuncSetAttribute(pass_c_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_ac));
    pass_c_kernel<V><<<blocks_ac, 256, smem_ac, s>>>(pp, nx, NL, NL, radices_of(p->ax[0]), twx, lpb, mode, NL);
    VIE_LAUNCH_CHECK();
  }
  return VIE_OK;
}

vie_status jm_matvec_impl(vie_plan* p, const void* x, void* y, int dtype, int mode, cudaStream_t s) {
  if (!p->jm_work || !p->Mjm64) {
    set_error("set the plan's permeability (vie_set_permeability) before applying the JM-VIE operator");
    return VIE_ERR_INVALID;
  }
  if (dtype == VIE_C64)
    return run_jm<float2>(p, (const float2*)x, (float2*)y, p->ghat32, p->chat32, p->Mjm32, p->ax[0].tw32,
                          p->ax[1].tw32, p->ax[2].tw32, mode, s);
  if (dtype == VIE_C128)
    return run_jm<double2>(p, (const double2*)x, (double2*)y, p->ghat64, p->chat64, p->Mjm64, p->ax[0].tw64,
                           p->ax[1].tw64, p->ax[2].tw64, mode, s);
  set_error("unknown dtype %d", dtype);
  return VIE_ERR_INVALID;
}

// The split pass B's buffer behind the x-pass spectra of a workspace of
// work_bytes, or null (that pass B is not needed or does not fit).
template <typename V>
static V* split_buffer(const vie_plan* p, V* work, size_t work_bytes) {
  const size_t xs = (size_t)3 * p->n[1] * p->n[2] * p->m[0];
  const size_t e = pass_b_split_elems(p->n[1], p->n[2], p->m[0], p->m[1], p->m[2]);
  if (e == 0 || (xs + e) * sizeof(V) > work_bytes) return nullptr;
  return work + xs;
}

template <typename V>
static vie_status run_one(vie_plan* p, const V* x, V* y, const V* ghat, const V* Mc, const V* twx, const V* twy,
                          const V* twz, int mode, V* work, size_t work_bytes, cudaStream_t s) {
  PassPtrs<V> pp;
  memset(&pp, 0, sizeof(pp));
  pp.x[0] = x;
  pp.y[0] = y;
  pp.work[0] = work;
  pp.work2[0] = split_buffer<V>(p, work, work_bytes);
  pp.ghat[0] = ghat;
  pp.M[0] = Mc;
  return run_passes<V>(p, pp, 1, twx, twy, twz, mode, s);
}

template <typename V>
static vie_status group_passes(vie_plan* const* plans, int count, const void* const* x, void* const* y, int mode,
                               cudaStream_t s, const int* const* live) {
  const vie_plan* p0 = plans[0];
  const bool f32 = sizeof(V) == sizeof(float2);
  const V* twx = f32 ? (const V*)p0->ax[0].tw32 : (const V*)p0->ax[0].tw64;
  const V* twy = f32 ? (const V*)p0->ax[1].tw32 : (const V*)p0->ax[1].tw64;
  const V* twz = f32 ? (const V*)p0->ax[2].tw32 : (const V*)p0->ax[2].tw64;
  for (int i0 = 0; i0 < count; i0 += kMaxBatch) {
    const int c = (count - i0) < kMaxBatch ? (count - i0) : kMaxBatch;
    PassPtrs<V> pp;
    memset(&pp, 0, sizeof(pp));
    for (int k = 0; k < c; ++k) {
      const vie_plan* q = plans[i0 + k];
      pp.x[k] = (const V*)x[i0 + k];
      pp.y[k] = (V*)y[i0 + k];
      pp.work[k] = (V*)q->work;
      pp.work2[k] = split_buffer<V>(q, (V*)q->work, q->work_bytes);
      pp.ghat[k] = f32 ? (const V*)q->ghat32 : (const V*)q->ghat64;
      pp.M[k] = f32 ? (const V*)q->M32 : (const V*)q->M64;
      pp.live[k] = live ? live[i0 + k] : nullptr;
    }
    vie_status st = run_passes<V>(p0, pp, c, twx, twy, twz, mode, s);
    if (st != VIE_OK) return st;
  }
  return VIE_OK;
}

vie_status matvec_group(vie_plan* const* plans, int count, const void* const* x, void* const* y, int dtype, int mode,
                        cudaStream_t s, const int* const* live) {
  if (dtype == VIE_C64) return group_passes<float2>(plans, count, x, y, mode, s, live);
  if (dtype == VIE_C128) return group_passes<double2>(plans, count, x, y, mode, s, live);
  set_error("unknown dtype %d", dtype);
  return VIE_ERR_INVALID;
}

vie_status matvec_impl(vie_plan* p, const void* x, void* y, int dtype, int mode, void* work, size_t work_bytes,
                       cudaStream_t s) {
  if (dtype == VIE_C64)
    return run_one<float2>(p, (const float2*)x, (float2*)y, p->ghat32, p->M32, p->ax[0].tw32, p->ax[1].tw32,
                           p->ax[2].tw32, mode, (float2*)work, work_bytes, s);
  if (dtype == VIE_C128)
    return run_one<double2>(p, (const double2*)x, (double2*)y, p->ghat64, p->M64, p->ax[0].tw64, p->ax[1].tw64,
                            p->ax[2].tw64, mode, (double2*)work, work_bytes, s);
  set_error("unknown dtype %d", dtype);
  return VIE_ERR_INVALID;
}

}  // namespace vie

// ---------------------------------------------------------------------------
// Operator application without any allocation by the library.
//
// Some callers cannot call cudaMalloc where they apply the operator: their
// device memory is owned by another allocator or held to a fixed budget after
// start-up, so they cannot create a second plan or a second workspace.  This
// variant runs the same three passes as vie_matvec, but its workspace is the
// file-scope array below instead of the plan's workspace, so it can run next
// to vie_matvec on the same plan without allocating anything.
//
// The array is part of the library image: every GPU that loads the library
// holds its kStaticScratchBytes until the process exits.  Host code cannot use
// the array's name as a device address (it names a host-side stand-in), so the
// device address is looked up with cudaGetSymbolAddress once per device, on
// the first call made while that device is current.
// ---------------------------------------------------------------------------
namespace vie {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
static void* g_static_scratch_addr[kMaxDevices] = {nullptr};

static vie_status static_scratch_address(void** out) {
  int dev = 0;
  VIE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d out of range for the static workspace", dev);
    return VIE_ERR_INVALID;
  }
  if (!g_static_scratch_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      set_error("cudaGetSymbolAddress of the static workspace failed: %s", cudaGetErrorString(e));
      return VIE_ERR_CUDA;
    }
    g_static_scratch_addr[dev] = ptr;
  }
  *out = g_static_scratch_addr[dev];
  return VIE_OK;
}

// Called by vie_plan_create and vie_plan_clone, where allocating is allowed:
// the lookup makes the runtime load this file's module (and with it the
// static array) on the current device, so that under lazy module loading the
// first vie_matvec_static_scratch call does not load it and reserve memory.
vie_status static_scratch_prepare() {
  void* unused = nullptr;
  return static_scratch_address(&unused);
}

}  // namespace vie

extern "C" vie_status vie_matvec_static_scratch(const vie_plan* plan, const void* x_dev, void* y_dev, int dtype,
                                                void* stream) {
  using namespace vie;
  clear_error();
  if (!plan || !x_dev || !y_dev) { set_error("null argument"); return VIE_ERR_INVALID; }
  if (dtype != VIE_C64 && dtype != VIE_C128) { set_error("dtype must be VIE_C64 or VIE_C128"); return VIE_ERR_INVALID; }
  const size_t vec_bytes = (size_t)3 * plan->n[0] * plan->n[1] * plan->n[2] * (dtype == VIE_C64 ? 8 : 16);
  const char* a = (const char*)x_dev;
  const char* b = (const char*)y_dev;
  if (a < b + vec_bytes && b < a + vec_bytes) { set_error("x and y overlap"); return VIE_ERR_INVALID; }
  const size_t need = (size_t)3 * plan->n[1] * plan->n[2] * plan->m[0] * (dtype == VIE_C64 ? 8 : 16);
  if (need > kStaticScratchBytes) {
    set_error("workspace of %zu bytes exceeds the static workspace of %zu bytes (3*ny*nz*Mx complex values)",
              need, kStaticScratchBytes);
    return VIE_ERR_INVALID;
  }
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != plan->device) {
    set_error("the plan's device (%d) must be current (current: %d)", plan->device, cur);
    return VIE_ERR_INVALID;
  }
  void* work = nullptr;
  vie_status st = static_scratch_address(&work);
  if (st != VIE_OK) return st;
  return matvec_impl(const_cast<vie_plan*>(plan), x_dev, y_dev, dtype, MODE_OPERATOR, work, kStaticScratchBytes,
                     (cudaStream_t)stream);
}
