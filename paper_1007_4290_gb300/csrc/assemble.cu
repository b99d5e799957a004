// Discretisation of the PML-stretched Helmholtz operator (Section 2.1, Eq. sigma,
// Eq. helmd) and the 5-point matrix-vector product y = A x, complex128.
#include "handle.h"

namespace {

// s(t) = 1 / (1 + i sigma(t)/omega), sigma of Eq. sigma; lo / hi: the layer at t = 0 /
// t = 1 is present (a side without it is a plain Dirichlet boundary, Section 2.5)
__device__ c128 stretch(double t, double eta, double pref, double omega, bool lo, bool hi) {
  double sig = 0.0;
  if (eta > 0.0) {
    if (t < eta) { if (lo) { double q = (t - eta) / eta; sig = pref * q * q; } }
    else if (t > 1.0 - eta) { if (hi) { double q = (t - 1.0 + eta) / eta; sig = pref * q * q; } }
  }
  return cinv(c128(1.0, sig / omega));
}

// One thread per node (i, j): the two edge coefficients east[j][i] (edge to the left
// of node i in row j) and north[j][i] (edge below node i), plus the node terms.  The
// right/upper boundary edges (index n) are written by the threads of the last column/row.
__global__ void assemble_kernel(int n, double h, double eta, double pref, double omega, int sides,
                                const double* __restrict__ c, c128* diag, c128* east,
                                c128* north, c128* s1s2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  if (i >= n || j >= n) return;
  double ih2 = 1.0 / (h * h);
  const bool l1 = sides & 1, h1 = sides & 2, l2 = sides & 4, h2 = sides & 8;
  c128 si = stretch((i + 1) * h, eta, pref, omega, l1, h1);       // s1 at node i
  c128 sj = stretch((j + 1) * h, eta, pref, omega, l2, h2);       // s2 at row j
  c128 sih_l = stretch((i + 0.5) * h, eta, pref, omega, l1, h1);  // half point i - 1/2
  c128 sih_r = stretch((i + 1.5) * h, eta, pref, omega, l1, h1);  // half point i + 1/2
  c128 sjh_l = stretch((j + 0.5) * h, eta, pref, omega, l2, h2);
  c128 sjh_r = stretch((j + 1.5) * h, eta, pref, omega, l2, h2);
  c128 inv_sj = cinv(sj), inv_si = cinv(si);
  c128 e_l = ih2 * (sih_l * inv_sj), e_r = ih2 * (sih_r * inv_sj);   // (s1/s2)_{i -+ 1/2, j}/h^2
  c128 n_l = ih2 * (sjh_l * inv_si), n_r = ih2 * (sjh_r * inv_si);   // (s2/s1)_{i, j -+ 1/2}/h^2
  long long p = (long long)j * n + i;
  east[(long long)j * (n + 1) + i] = e_l;
  if (i == n - 1) east[(long long)j * (n + 1) + n] = e_r;
  north[(long long)j * n + i] = n_l;
  if (j == n - 1) north[(long long)n * n + i] = n_r;
  c128 ss = si * sj;
  if (s1s2) s1s2[p] = ss;
  double cc = c[p];
  c128 k2 = (omega * omega / (cc * cc)) * cinv(ss);
  diag[p] = k2 - (((e_l + e_r) + n_l) + n_r);
}

// y[s] = A x[s] (f null) or the residual y[s] = f[s] - A x[s], for right-hand sides
// s0 .. s0 + 7: one thread per node, the five coefficients loaded once (negated for the
// residual), the 8 x 5 neighbour values of all eight right-hand sides in flight together
constexpr int kMvRhs = 8;
template <typename T>
__global__ void matvec_kernel(int n, long long N, int nrhs, const c128* __restrict__ diag,
                              const c128* __restrict__ east, const c128* __restrict__ north,
                              const c128* __restrict__ x, c128* __restrict__ y, const c128* __restrict__ f) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int j = (int)(p / n), i = (int)(p - (long long)j * n);
  const int s0 = blockIdx.y * kMvRhs;
  const c128 zero(0.0, 0.0);
  const T sg = f ? T(-1) : T(1);
  const Cx<T> d = sg * cvt<T>(diag[p]);
  const Cx<T> el = sg * cvt<T>(i > 0 ? east[(long long)j * (n + 1) + i] : zero);
  const Cx<T> er = sg * cvt<T>(i < n - 1 ? east[(long long)j * (n + 1) + i + 1] : zero);
  const Cx<T> nl = sg * cvt<T>(j > 0 ? north[(long long)j * n + i] : zero);
  const Cx<T> nr = sg * cvt<T>(j < n - 1 ? north[(long long)(j + 1) * n + i] : zero);
  const long long pl = i > 0 ? p - 1 : p, pr = i < n - 1 ? p + 1 : p;
  const long long pd = j > 0 ? p - n : p, pu = j < n - 1 ? p + n : p;
  Cx<T> v[kMvRhs][5];
#pragma unroll
  for (int u = 0; u < kMvRhs; ++u) {
    if (s0 + u < nrhs) {
      const c128* xs = x + (long long)(s0 + u) * N;
      v[u][0] = cvt<T>(xs[p]);
      v[u][1] = cvt<T>(xs[pl]);
      v[u][2] = cvt<T>(xs[pr]);
      v[u][3] = cvt<T>(xs[pd]);
      v[u][4] = cvt<T>(xs[pu]);
    }
  }
  // away from the PML every coefficient is real: complex x real multiply-adds give the
  // same values with half the FP64 operations (FP64 throughput bounds this kernel)
  const bool real_coef = d.im == 0.0 && el.im == 0.0 && er.im == 0.0 && nl.im == 0.0 && nr.im == 0.0;
  if (real_coef) {
#pragma unroll
    for (int u = 0; u < kMvRhs; ++u) {
      if (s0 + u < nrhs) {
        const Cx<T> f0 = f ? cvt<T>(f[(long long)(s0 + u) * N + p]) : Cx<T>(0, 0);
        T re = fma(d.re, v[u][0].re, f0.re), im = fma(d.re, v[u][0].im, f0.im);
        re = fma(el.re, v[u][1].re, re); im = fma(el.re, v[u][1].im, im);
        re = fma(er.re, v[u][2].re, re); im = fma(er.re, v[u][2].im, im);
        re = fma(nl.re, v[u][3].re, re); im = fma(nl.re, v[u][3].im, im);
        re = fma(nr.re, v[u][4].re, re); im = fma(nr.re, v[u][4].im, im);
        y[(long long)(s0 + u) * N + p] = c128(re, im);
      }
    }
    return;
  }
#pragma unroll
  for (int u = 0; u < kMvRhs; ++u) {
    if (s0 + u < nrhs) {
      Cx<T> acc = f ? cvt<T>(f[(long long)(s0 + u) * N + p]) : Cx<T>(0, 0);
      cfma(acc, d, v[u][0]);
      cfma(acc, el, v[u][1]);
      cfma(acc, er, v[u][2]);
      cfma(acc, nl, v[u][3]);
      cfma(acc, nr, v[u][4]);
      y[(long long)(s0 + u) * N + p] = cvt<double>(acc);
    }
  }
}

}  // namespace

int hsw_assemble(hsweep_s* h, double pml_C, int pml_form, int pml_sides, c128* diag, c128* east, c128* north,
                 c128* s1s2) {
  double eta = h->pml_width * h->h;
  double pref = (pml_form == 0 && eta > 0) ? pml_C / eta : pml_C;
  dim3 grid(div_up(h->n, 128), h->n);
  assemble_kernel<<<grid, 128, 0, h->stream>>>(h->n, h->h, eta, pref, h->omega, pml_sides, h->d_c, diag, east, north,
                                                s1s2);
  h->nlaunch += 1;
  HSW_CUDA(cudaGetLastError());
  return HSWEEP_OK;
}

static int matvec_launch(hsweep_s* h, const c128* x, c128* y, const c128* f, int nrhs, bool lowp) {
  if (nrhs <= 0) return HSWEEP_OK;
  dim3 grid(div_up(h->N, 256), div_up(nrhs, kMvRhs));
  if (lowp)
    matvec_kernel<float><<<grid, 256, 0, h->stream>>>(h->n, (long long)h->N, nrhs, h->d_diag, h->d_east,
                                                      h->d_north, x, y, f);
  else
    matvec_kernel<double><<<grid, 256, 0, h->stream>>>(h->n, (long long)h->N, nrhs, h->d_diag, h->d_east,
                                                       h->d_north, x, y, f);
  h->nlaunch += 1;
  HSW_CUDA(cudaGetLastError());
  return HSWEEP_OK;
}

int hsw_matvec_prec(hsweep_s* h, const c128* x, c128* y, int nrhs, bool lowp) {
  return matvec_launch(h, x, y, nullptr, nrhs, lowp);
}

int hsw_matvec(hsweep_s* h, const c128* x, c128* y, int nrhs) { return matvec_launch(h, x, y, nullptr, nrhs, false); }

int hsw_residual(hsweep_s* h, const c128* f, const c128* u, c128* r, int nrhs) {
  return matvec_launch(h, u, r, f, nrhs, false);
}

namespace {

// f[s][node next to the side, k] -= (edge coefficient to the boundary) * b[s][k]
__global__ void boundary_rhs_kernel(int n, long long N, int nrhs, int side, int dir, const c128* __restrict__ east,
                                    const c128* __restrict__ north, const c128* __restrict__ b,
                                    c128* __restrict__ f) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)nrhs * n) return;
  const int s = (int)(e / n), k = (int)(e - (long long)s * n);
  const int jint = dir > 0 ? k : n - 1 - k;     // handle row of caller row k
  long long p;
  c128 coef;
  switch (side) {
    case 0: p = (long long)k * n; coef = east[(long long)jint * (n + 1)]; break;
    case 1: p = (long long)k * n + n - 1; coef = east[(long long)jint * (n + 1) + n]; break;
    case 2: p = k; coef = north[(long long)(dir > 0 ? 0 : n) * n + k]; break;
    default: p = (long long)(n - 1) * n + k; coef = north[(long long)(dir > 0 ? n : 0) * n + k]; break;
  }
  c128 v = f[(long long)s * N + p];
  cfma(v, -coef, b[(long long)s * n + k]);
  f[(long long)s * N + p] = v;
}

}  // namespace

int hsw_boundary_rhs(hsweep_s* h, int side, const c128* b, c128* f, int nrhs) {
  if (nrhs <= 0) return HSWEEP_OK;
  const long long work = (long long)nrhs * h->n;
  boundary_rhs_kernel<<<div_up(work, 256), 256, 0, h->stream>>>(h->n, (long long)h->N, nrhs, side, h->dir, h->d_east,
                                                                h->d_north, b, f);
  h->nlaunch += 1;
  HSW_CUDA(cudaGetLastError());
  return HSWEEP_OK;
}
