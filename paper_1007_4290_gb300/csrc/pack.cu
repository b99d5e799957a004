// Leaf-major packing of the H-factors for the sweep.
//
// For layer m and leaf lam (rows [lo, lo + s) of the layer) the record is
//   [ D_lam, leaf x leaf, row-major ]
//   [ for depth d = 1..L: the s rows of F_v (v = ancestor of lam at depth d),
//     row-major with an odd row stride rs_d >= rank(v) (zero padding) ]
// rounded up to an even number of entries (16-byte multiple).  Records are stored in
// leaf order, so the rows of every subtree (a sweep CTA's slab) are one contiguous
// range, fetched by a single bulk copy.  The odd row stride keeps row-parallel shared-
// memory reads free of bank conflicts.
#include <algorithm>
#include "handle.h"

namespace {

__host__ __device__ __forceinline__ int row_stride(int r) { return r == 0 ? 0 : (r | 1); }

template <typename R>
__global__ void pack_layers(int m0, int n, int L, int leaf, int nnodes, const int* __restrict__ lo,
                            const int* __restrict__ sz, const long long* __restrict__ off,
                            const Cx<R>* __restrict__ fac, long long layer_stride, const int* __restrict__ rank,
                            Cx<R>* __restrict__ pack, long long pack_stride, long long* __restrict__ recoff) {
  extern __shared__ long long sizes[];   // [nleaves + 1]
  const int m = m0 + blockIdx.x;
  const int nleaves = 1 << L;
  const int* rk = rank + (long long)m * nnodes;
  for (int j = threadIdx.x; j < nleaves; j += blockDim.x) {
    const int lam = nleaves + j, s = sz[lam];
    long long e = (long long)leaf * leaf;
    for (int d = 1; d <= L; ++d) e += (long long)s * row_stride(rk[lam >> (L - d)]);
    sizes[j] = (e + 1) & ~1LL;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long acc = 0;
    for (int j = 0; j < nleaves; ++j) { long long t = sizes[j]; sizes[j] = acc; acc += t; }
    sizes[nleaves] = acc;
  }
  __syncthreads();
  long long* ro = recoff + (long long)m * (nleaves + 1);
  for (int j = threadIdx.x; j <= nleaves; j += blockDim.x) ro[j] = sizes[j];
  const Cx<R>* F = fac + (long long)m * layer_stride;
  Cx<R>* P = pack + (long long)m * pack_stride;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j < nleaves; j += nw) {
    const int lam = nleaves + j, s = sz[lam], l0 = lo[lam];
    long long o = sizes[j];
    const long long end = sizes[j + 1];
    for (int e = lane; e < leaf * leaf; e += 32) {       // column-major store -> row-major
      const int a = e / leaf, b = e % leaf;
      P[o + e] = F[(long long)j * leaf * leaf + b * leaf + a];
    }
    o += (long long)leaf * leaf;
    for (int d = 1; d <= L; ++d) {
      const int v = lam >> (L - d);
      const int r = rk[v], rs = row_stride(r), sv = sz[v], ro_v = l0 - lo[v];
      const Cx<R>* Fv = F + off[v];
      for (int e = lane; e < s * rs; e += 32) {
        const int a = e / rs, k = e % rs;
        P[o + e] = k < r ? Fv[(long long)k * sv + ro_v + a] : Cx<R>(0, 0);
      }
      o += (long long)s * rs;
    }
    for (long long e = o + lane; e < end; e += 32) P[e] = Cx<R>(0, 0);
  }
}

}  // namespace

int hsw_pack(hsweep_s* h, int m0, int m1) {
  if (m1 <= m0) return HSWEEP_OK;
  const size_t smem = (size_t)(h->nleaves + 1) * sizeof(long long);
  if (smem > 48 * 1024) return HSWEEP_ERR_ARG;
  if (h->prec == HSWEEP_FP64)
    pack_layers<double><<<m1 - m0, 256, smem, h->stream>>>(m0, h->n, h->L, h->leaf, h->nnodes, h->d_lo, h->d_sz,
        h->d_off, (const c128*)h->d_fac, h->layer_stride, h->d_rank, (c128*)h->d_pack, h->pack_stride, h->d_recoff);
  else
    pack_layers<float><<<m1 - m0, 256, smem, h->stream>>>(m0, h->n, h->L, h->leaf, h->nnodes, h->d_lo, h->d_sz,
        h->d_off, (const c64*)h->d_fac, h->layer_stride, h->d_rank, (c64*)h->d_pack, h->pack_stride, h->d_recoff);
  h->nlaunch += 1;
  HSW_CUDA(cudaGetLastError());
  // largest slab record per slab depth, and the largest rank, for the sweep's
  // shared-memory plan
  std::vector<long long> ro((size_t)h->n * (h->nleaves + 1));
  std::vector<int> rk((size_t)h->n * h->nnodes);
  HSW_CUDA(cudaMemcpyAsync(ro.data(), h->d_recoff, ro.size() * sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
  HSW_CUDA(cudaMemcpyAsync(rk.data(), h->d_rank, rk.size() * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  HSW_CUDA(cudaStreamSynchronize(h->stream));
  const size_t es = h->fac_elem();
  h->slab_bytes_max.assign(h->L + 1, 0);
  h->team_plans.clear();
  for (int dC = 0; dC <= h->L; ++dC) {
    const int nl = 1 << (h->L - dC);
    long long mx = 0;
    for (int m = 0; m < h->n; ++m) {
      const long long* r = ro.data() + (size_t)m * (h->nleaves + 1);
      for (int c = 0; c < (1 << dC); ++c) mx = std::max(mx, r[(c + 1) * nl] - r[c * nl]);
    }
    h->slab_bytes_max[dC] = mx * (long long)es;
  }
  h->rank_max = 0;
  for (int v : rk) h->rank_max = std::max(h->rank_max, v);
  h->rank_max_depth.assign(h->L + 1, 0);
  for (int m = 0; m < h->n; ++m)
    for (int v = 2; v < h->nnodes; ++v) {
      int d = 0;
      while ((2 << d) <= v) ++d;
      h->rank_max_depth[d] = std::max(h->rank_max_depth[d], rk[(size_t)m * h->nnodes + v]);
    }
  h->pack_valid = true;
  return HSWEEP_OK;
}
