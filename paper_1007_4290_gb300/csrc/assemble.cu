// Discretisation of the PML-stretched Helmholtz operator (Section 2.1, Eq. sigma,
// Eq. helmd) and the 5-point matrix-vector product y = A x, complex128.
#include "handle.h"

namespace {

// s(t) = 1 / (1 + i sigma(t)/omega), sigma of Eq. sigma.
__device__ c128 stretch(double t, double eta, double pref, double omega) {
  double sig = 0.0;
  if (eta > 0.0) {
    if (t < eta) { double q = (t - eta) / eta; sig = pref * q * q; }
    else if (t > 1.0 - eta) { double q = (t - 1.0 + eta) / eta; sig = pref * q * q; }
  }
  return cinv(c128(1.0, sig / omega));
}

// One thread per node (i, j): the two edge coefficients east[j][i] (edge to the left
// of node i in row j) and north[j][i] (edge below node i), plus the node terms.  The
// right/upper boundary edges (index n) are written by the threads of the last column/row.
__global__ void assemble_kernel(int n, double h, double eta, double pref, double omega,
                                const double* __restrict__ c, c128* diag, c128* east,
                                c128* north, c128* s1s2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  if (i >= n || j >= n) return;
  double ih2 = 1.0 / (h * h);
  c128 si = stretch((i + 1) * h, eta, pref, omega);       // s1 at node i
  c128 sj = stretch((j + 1) * h, eta, pref, omega);       // s2 at row j
  c128 sih_l = stretch((i + 0.5) * h, eta, pref, omega);  // half point i - 1/2
  c128 sih_r = stretch((i + 1.5) * h, eta, pref, omega);  // half point i + 1/2
  c128 sjh_l = stretch((j + 0.5) * h, eta, pref, omega);
  c128 sjh_r = stretch((j + 1.5) * h, eta, pref, omega);
  c128 inv_sj = cinv(sj), inv_si = cinv(si);
  c128 e_l = ih2 * (sih_l * inv_sj), e_r = ih2 * (sih_r * inv_sj);   // (s1/s2)_{i -+ 1/2, j}/h^2
  c128 n_l = ih2 * (sjh_l * inv_si), n_r = ih2 * (sjh_r * inv_si);   // (s2/s1)_{i, j -+ 1/2}/h^2
  long long p = (long long)j * n + i;
  east[(long long)j * (n + 1) + i] = e_l;
  if (i == n - 1) east[(long long)j * (n + 1) + n] = e_r;
  north[(long long)j * n + i] = n_l;
  if (j == n - 1) north[(long long)n * n + i] = n_r;
  c128 ss = si * sj;
  s1s2[p] = ss;
  double cc = c[p];
  c128 k2 = (omega * omega / (cc * cc)) * cinv(ss);
  diag[p] = k2 - (((e_l + e_r) + n_l) + n_r);
}

__global__ void matvec_kernel(int n, long long N, int nrhs, const c128* __restrict__ diag,
                              const c128* __restrict__ east, const c128* __restrict__ north,
                              const c128* __restrict__ x, c128* __restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  if (i >= n) return;
  long long p = (long long)j * n + i;
  c128 d = diag[p];
  c128 el = east[(long long)j * (n + 1) + i], er = east[(long long)j * (n + 1) + i + 1];
  c128 nl = north[(long long)j * n + i], nr = north[(long long)(j + 1) * n + i];
  for (int s = blockIdx.z; s < nrhs; s += gridDim.z) {
    const c128* xs = x + s * N;
    c128 acc = d * xs[p];
    if (i > 0) cfma(acc, el, xs[p - 1]);
    if (i < n - 1) cfma(acc, er, xs[p + 1]);
    if (j > 0) cfma(acc, nl, xs[p - n]);
    if (j < n - 1) cfma(acc, nr, xs[p + n]);
    y[s * N + p] = acc;
  }
}

}  // namespace

int hsw_assemble(hsweep_s* h, double pml_C, int pml_form) {
  double eta = h->pml_width * h->h;
  double pref = (pml_form == 0 && eta > 0) ? pml_C / eta : pml_C;
  dim3 grid(div_up(h->n, 128), h->n);
  assemble_kernel<<<grid, 128, 0, h->stream>>>(h->n, h->h, eta, pref, h->omega, h->d_c,
                                                h->d_diag, h->d_east, h->d_north, h->d_s1s2);
  h->nlaunch += 1;
  HSW_CUDA(cudaGetLastError());
  return HSWEEP_OK;
}

int hsw_matvec(hsweep_s* h, const c128* x, c128* y, int nrhs) {
  if (nrhs <= 0) return HSWEEP_OK;
  dim3 grid(div_up(h->n, 128), h->n, nrhs < 8 ? nrhs : 8);
  matvec_kernel<<<grid, 128, 0, h->stream>>>(h->n, (long long)h->N, nrhs, h->d_diag, h->d_east,
                                              h->d_north, x, y);
  h->nlaunch += 1;
  HSW_CUDA(cudaGetLastError());
  return HSWEEP_OK;
}
