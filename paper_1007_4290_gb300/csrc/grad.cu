// Misfit J = 1/2 sum_s ||R u_s - d_s||^2 and its gradient with respect to c, by the
// adjoint method with the same factorisation.  A(c) is complex symmetric (A^t = A,
// Section 2.1), so the adjoint system A^H lambda = b is solved as
//     lambda = conj(A^{-1} conj(b)).
// Only the diagonal of A depends on c (Eq. helmd): dA_ii/dc_i = -2 omega^2 / ((s1 s2)_i c_i^3),
// hence dJ/dc_i = sum_s Re(conj(lambda_{s,i}) dA_ii/dc_i u_{s,i})
//              = -2 omega^2 c_i^{-3} sum_s Re(v_{s,i} u_{s,i} / (s1 s2)_i),  v_s = conj(lambda_s).
#include <vector>
#include "handle.h"

namespace {

// res[s][k] = u_s[rec_k] - d[s][k]; partial misfit per RHS
__global__ void receiver_residual(const c128* __restrict__ U, long long N, const int* __restrict__ rec, int nrec,
                                  const c128* __restrict__ d, c128* __restrict__ res, double* __restrict__ jpart) {
  const int s = blockIdx.x;
  __shared__ double red[32];
  double acc = 0;
  for (int k = threadIdx.x; k < nrec; k += blockDim.x) {
    c128 r = U[s * N + rec[k]] - d[(long long)s * nrec + k];
    res[(long long)s * nrec + k] = r;
    acc += abs2(r);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    jpart[s] = 0.5 * t;
  }
}

// B_s = conj(-R^t res_s): scatter (duplicated receivers accumulate)
__global__ void adjoint_rhs(const c128* __restrict__ res, const int* __restrict__ rec, int nrec, long long N,
                            c128* __restrict__ B) {
  const int s = blockIdx.y;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nrec; k += gridDim.x * blockDim.x) {
    c128 r = res[(long long)s * nrec + k];
    double* p = reinterpret_cast<double*>(B + s * N + rec[k]);
    atomicAdd(p, -r.re);
    atomicAdd(p + 1, r.im);
  }
}

__global__ void gradient_kernel(const c128* __restrict__ U, const c128* __restrict__ V, int nsrc, long long N,
                                const double* __restrict__ c, const c128* __restrict__ s1s2, double omega,
                                double* __restrict__ g) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    c128 sum(0, 0);
    for (int s = 0; s < nsrc; ++s) sum += V[s * N + i] * U[s * N + i];
    c128 q = sum * cinv(s1s2[i]);
    const double ci = c[i];
    g[i] = -2.0 * omega * omega / (ci * ci * ci) * q.re;
  }
}

}  // namespace

int hsw_grad(hsweep_s* h, const c128* f, int nsrc, const int* rec, int nrec, const c128* d, double* grad,
             double* misfit, double tol) {
  const long long N = h->N;
  c128 *U = nullptr, *B = nullptr, *V = nullptr, *res = nullptr;
  double* jpart = nullptr;
  int rc;
  auto cleanup = [&]() {
    hsw_release(h, U); hsw_release(h, B); hsw_release(h, V); hsw_release(h, res); hsw_release(h, jpart);
  };
#define A(p, bytes) do { rc = hsw_alloc(h, (void**)&(p), (size_t)(bytes)); if (rc) { cleanup(); return rc; } } while (0)
  A(U, (size_t)nsrc * N * sizeof(c128));
  A(B, (size_t)nsrc * N * sizeof(c128));
  A(V, (size_t)nsrc * N * sizeof(c128));
  A(res, (size_t)nsrc * nrec * sizeof(c128));
  A(jpart, (size_t)nsrc * sizeof(double));
#undef A
  // receivers must be valid node offsets
  {
    std::vector<int> hr(nrec);
    if (cudaMemcpy(hr.data(), rec, nrec * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) { cleanup(); return HSWEEP_ERR_CUDA; }
    for (int k = 0; k < nrec; ++k)
      if (hr[k] < 0 || hr[k] >= N) { cleanup(); return HSWEEP_ERR_ARG; }
  }
  std::vector<int> it(nsrc);
  std::vector<double> rr(nsrc);
  if (cudaMemsetAsync(U, 0, (size_t)nsrc * N * sizeof(c128), h->stream) != cudaSuccess) { cleanup(); return HSWEEP_ERR_CUDA; }
  rc = hsw_solve(h, f, U, nsrc, tol, it.data(), rr.data());
  if (rc != HSWEEP_OK) { cleanup(); return rc; }
  receiver_residual<<<nsrc, 256, 0, h->stream>>>(U, N, rec, nrec, d, res, jpart);
  h->nlaunch += 1;
  if (cudaGetLastError() != cudaSuccess) { cleanup(); return HSWEEP_ERR_CUDA; }
  if (cudaMemsetAsync(B, 0, (size_t)nsrc * N * sizeof(c128), h->stream) != cudaSuccess) { cleanup(); return HSWEEP_ERR_CUDA; }
  adjoint_rhs<<<dim3((nrec + 255) / 256, nsrc), 256, 0, h->stream>>>(res, rec, nrec, N, B);
  h->nlaunch += 1;
  if (cudaGetLastError() != cudaSuccess) { cleanup(); return HSWEEP_ERR_CUDA; }
  if (cudaMemsetAsync(V, 0, (size_t)nsrc * N * sizeof(c128), h->stream) != cudaSuccess) { cleanup(); return HSWEEP_ERR_CUDA; }
  rc = hsw_solve(h, B, V, nsrc, tol, it.data(), rr.data());
  if (rc != HSWEEP_OK) { cleanup(); return rc; }
  gradient_kernel<<<1216, 256, 0, h->stream>>>(U, V, nsrc, N, h->d_c, h->d_s1s2, h->omega, grad);
  h->nlaunch += 1;
  if (cudaGetLastError() != cudaSuccess) { cleanup(); return HSWEEP_ERR_CUDA; }
  std::vector<double> hj(nsrc);
  if (cudaMemcpyAsync(hj.data(), jpart, nsrc * sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cleanup();
    return HSWEEP_ERR_CUDA;
  }
  double J = 0;
  for (double v : hj) J += v;
  if (misfit) *misfit = J;
  cleanup();
  return HSWEEP_OK;
}
