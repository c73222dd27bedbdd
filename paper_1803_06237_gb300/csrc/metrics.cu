// Field on the centre axis and the reflection coefficient R (Sec. 5.1 of
// arXiv:1803.06237): E = J / (c_e chi) from the equivalent current of Sec. 3,
// taken on the voxel row (ny/2, nz/2), and
// R = sum |E_ref - E|^2 / sum |E_ref|^2 over the axis voxels before the
// absorber.  The common factor c_e h^(3/2) cancels in R and is not applied.
#include "vie_internal.cuh"

namespace vie {

__global__ void axis_field_kernel(const double2* __restrict__ w, const double2* __restrict__ chi, int nx, int ny,
                                  int nz, int n_keep, double2* __restrict__ out, int* __restrict__ bad) {
  const size_t N = (size_t)nx * ny * nz;
  const int yc = ny / 2, zc = nz / 2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n_keep; i += gridDim.x * blockDim.x) {
    const int c = i / n_keep, ix = i - c * n_keep;
    const size_t v = ((size_t)zc * ny + yc) * nx + ix;
    const double2 a = w[c * N + v], d = chi[v];
    const double den = d.x * d.x + d.y * d.y;
    if (den == 0.0) {
      atomicExch(bad, 1);
      out[i] = make_double2(0.0, 0.0);
    } else {
      out[i] = make_double2((a.x * d.x + a.y * d.y) / den, (a.y * d.x - a.x * d.y) / den);
    }
  }
}

// one block: sums in FP64, fixed order per thread then a tree
__global__ void reflection_kernel(const double2* __restrict__ Eref, const double2* __restrict__ E, int count,
                                  double* __restrict__ out) {
  __shared__ double sn[256], sd[256];
  double num = 0.0, den = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const double2 r = Eref[i], e = E[i];
    const double dx = r.x - e.x, dy = r.y - e.y;
    num += dx * dx + dy * dy;
    den += r.x * r.x + r.y * r.y;
  }
  sn[threadIdx.x] = num;
  sd[threadIdx.x] = den;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sn[threadIdx.x] += sn[threadIdx.x + s];
      sd[threadIdx.x] += sd[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sn[0];
    out[1] = sd[0];
  }
}

// Transmission through a voxel plane (Sec. 5.2): T = sum over the voxels of
// plane ix with chi != 0 of |E|^2, E = J / (c_e chi), all three components
// (the common factor |c_e|^2 h^3 is not applied).  One block, FP64 sums in a
// fixed order.
__global__ void slice_power_kernel(const double2* __restrict__ w, const double2* __restrict__ chi, int nx, int ny,
                                   int nz, int ix, double* __restrict__ out) {
  __shared__ double sp[256];
  const size_t N = (size_t)nx * ny * nz;
  double acc = 0.0;
  for (int i = threadIdx.x; i < 3 * ny * nz; i += blockDim.x) {
    const int c = i / (ny * nz), yz = i - c * ny * nz;
    const size_t v = (size_t)yz * nx + ix;
    const double2 d = chi[v];
    const double den = d.x * d.x + d.y * d.y;
    if (den == 0.0) continue;
    const double2 a = w[c * N + v];
    acc += (a.x * a.x + a.y * a.y) / den;
  }
  sp[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sp[threadIdx.x] += sp[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sp[0];
}

}  // namespace vie

using namespace vie;

extern "C" vie_status vie_slice_power(const vie_plan* p, const void* w_dev, int ix, double* t_out, void* stream) {
  clear_error();
  if (!p || !w_dev || !t_out) { set_error("null argument"); return VIE_ERR_INVALID; }
  if (ix < 0 || ix >= p->n[0]) { set_error("ix must be in [0, nx)"); return VIE_ERR_INVALID; }
  cudaStream_t s = (cudaStream_t)stream;
  double* d = nullptr;
  VIE_CUDA_TRY(cudaMallocAsync((void**)&d, sizeof(double), s));
  slice_power_kernel<<<1, 256, 0, s>>>((const double2*)w_dev, p->chi64, p->n[0], p->n[1], p->n[2], ix, d);
  VIE_LAUNCH_CHECK();
  double h = 0.0;
  VIE_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, s));
  VIE_CUDA_TRY(cudaFreeAsync(d, s));
  VIE_CUDA_TRY(cudaStreamSynchronize(s));
  *t_out = h;
  return VIE_OK;
}

extern "C" vie_status vie_axis_field(const vie_plan* p, const void* w_dev, int n_keep, void* e_dev, void* stream) {
  clear_error();
  if (!p || !w_dev || !e_dev) { set_error("null argument"); return VIE_ERR_INVALID; }
  if (n_keep < 1 || n_keep > p->n[0]) { set_error("n_keep must be in [1, nx]"); return VIE_ERR_INVALID; }
  cudaStream_t s = (cudaStream_t)stream;
  int* bad = nullptr;
  VIE_CUDA_TRY(cudaMallocAsync((void**)&bad, sizeof(int), s));
  VIE_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
  axis_field_kernel<<<(3 * n_keep + 255) / 256, 256, 0, s>>>((const double2*)w_dev, p->chi64, p->n[0], p->n[1],
                                                              p->n[2], n_keep, (double2*)e_dev, bad);
  VIE_LAUNCH_CHECK();
  int hbad = 0;
  VIE_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  VIE_CUDA_TRY(cudaFreeAsync(bad, s));
  VIE_CUDA_TRY(cudaStreamSynchronize(s));
  if (hbad) { set_error("chi = 0 on the axis: the field is undefined there"); return VIE_ERR_NONFINITE; }
  return VIE_OK;
}

extern "C" vie_status vie_reflection(const void* eref_dev, const void* e_dev, int count, double* r_out, void* stream) {
  clear_error();
  if (!eref_dev || !e_dev || !r_out || count < 1) { set_error("null argument or count < 1"); return VIE_ERR_INVALID; }
  cudaStream_t s = (cudaStream_t)stream;
  double* d = nullptr;
  VIE_CUDA_TRY(cudaMallocAsync((void**)&d, 2 * sizeof(double), s));
  reflection_kernel<<<1, 256, 0, s>>>((const double2*)eref_dev, (const double2*)e_dev, count, d);
  VIE_LAUNCH_CHECK();
  double h[2] = {0.0, 0.0};
  VIE_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
  VIE_CUDA_TRY(cudaFreeAsync(d, s));
  VIE_CUDA_TRY(cudaStreamSynchronize(s));
  if (h[1] == 0.0) { set_error("reference field is zero"); return VIE_ERR_NONFINITE; }
  *r_out = h[0] / h[1];
  return VIE_OK;
}
