// Sweep direction (Section 3.1, the dependence on the sweeping direction): the sweep runs
// over the layers in the order x2 = 0 upward (Algorithms 2.5/2.6) or, with
// sweep_dir = -1, from x2 = 1 downward.  The downward sweep of A is the upward sweep of
// the reflected problem: with P the reversal of the layer order, the 5-point operator of
// the velocity P c is P A P (the grid, the PML and the coefficients are symmetric under
// x2 -> 1 - x2), so a handle with sweep_dir = -1 factors P A P and the public calls map
// their vectors through P on the way in and out.
#include "handle.h"

namespace {

// out[s][m][i] = in[s][n - 1 - m][i] for s < nvec (layers of n entries each)
template <typename T>
__global__ void flip_layers(const T* __restrict__ in, T* __restrict__ out, int n, long long N, int nvec) {
  const long long tot = (long long)nvec * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long s = e / N, p = e - s * N;
    const long long m = p / n, i = p - m * n;
    out[e] = in[s * N + (n - 1 - m) * n + i];
  }
}

// node indices of the reflected grid: p = m n + i -> (n - 1 - m) n + i; out of range
// indices are kept (the callee rejects them)
__global__ void flip_index(const int* __restrict__ in, int* __restrict__ out, int n, long long N, int cnt) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
    const int p = in[e];
    out[e] = (p >= 0 && p < N) ? (n - 1 - p / n) * n + p % n : p;
  }
}

unsigned flip_grid(long long work) {
  long long b = (work + 255) / 256;
  return (unsigned)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

}  // namespace

int hsw_flip_reserve(hsweep_s* h, size_t bytes) {
  if (bytes <= h->flip_cap) return HSWEEP_OK;
  int rc = hsw_regrow(h, &h->d_flip, bytes);
  if (rc) {
    if (!h->d_flip) h->flip_cap = 0;
    return rc;
  }
  h->flip_cap = bytes;
  return HSWEEP_OK;
}

int hsw_flip_c128(hsweep_s* h, const c128* in, c128* out, int nvec) {
  if (nvec <= 0) return HSWEEP_OK;
  flip_layers<c128><<<flip_grid((long long)nvec * h->N), 256, 0, h->stream>>>(in, out, h->n, h->N, nvec);
  h->nlaunch += 1;
  HSW_CUDA(cudaGetLastError());
  return HSWEEP_OK;
}

int hsw_flip_real(hsweep_s* h, const double* in, double* out) {
  flip_layers<double><<<flip_grid(h->N), 256, 0, h->stream>>>(in, out, h->n, h->N, 1);
  h->nlaunch += 1;
  HSW_CUDA(cudaGetLastError());
  return HSWEEP_OK;
}

int hsw_flip_index(hsweep_s* h, const int* in, int* out, int cnt) {
  if (cnt <= 0) return HSWEEP_OK;
  flip_index<<<flip_grid(cnt), 256, 0, h->stream>>>(in, out, h->n, h->N, cnt);
  h->nlaunch += 1;
  HSW_CUDA(cudaGetLastError());
  return HSWEEP_OK;
}
