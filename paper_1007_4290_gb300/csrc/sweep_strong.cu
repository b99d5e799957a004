// The apply z = M r of Algorithm 2.6 on strongly admissible T~_m (Section 2.3, the
// strongly admissible case), read in their own format instead of the expanded
// sibling-pair store.
//
// Format.  Per layer m, one record per leaf in leaf order; the layout is the same for
// every layer.  Leaf lam has s rows, its neighbouring leaves sl (left) and sr (right) rows
// (0 at the ends of the layer); its rows have stride rs = (s + sl + sr + 3 R (L - 1)) | 1
// and row i holds
//     [ T(lam, lam)[i, :] | T(lam, lam - 1)[i, :] | T(lam, lam + 1)[i, :] |
//       for d = 2..L and t = 0, 1, 2: W_{v_d, t}[i_v, 0..R) ]
// with v_d the ancestor of lam at depth d and i_v the row's index in v_d.  The
// interaction list of the cluster with index c at depth d (0-based from the left) is
// c - 2, c + 2, c + 3 for even c and c - 3, c - 2, c + 2 for odd c (those inside the
// layer), slot t in that order.  A well-separated pair (u, w) is T(u, w) = W_{u,t(w)}
// W_{w,t(u)}^t, and by the symmetry of T~_m, T(w, u) = W_{w,t(u)} W_{u,t(w)}^t.  Entries of
// missing partners are zero.  A row holds 3 leaf + 3 R (L - 1) entries (60 at n = 1023,
// R = 2) against leaf + the expanded ranks 3 R (L - d) + leaf summed over d in the
// sibling-pair store (about 190).  The records are written by the setup from the exact
// strongly admissible factors, before the recompression that the setup's own arithmetic
// needs (setup.cu), so this apply uses the strongly admissible T~_m exactly.
//
// Kernel.  Teams of C = 2^dC CTAs as in sweep_team.cu (cooperative launch, one slab of
// rows per CTA, G right-hand sides per team, 2n - 1 dependent steps).  One step:
//   0. the slab's record of the layer is in shared memory (bulk copy issued a step ahead);
//      the rows of the slab's first and last leaves are published (the neighbours' near
//      field);
//   1. reductions q_{v,t} = W_{v,t}^t x over the slab's rows for every cluster v at depth
//      >= 2 that meets the slab (partial sums for the ancestors at depths <= dC), published
//      to L2 with the step's tag;
//   2. the gather: for the ancestors, the partners' sums over the CTAs that hold them; for
//      the slab's own clusters, the sums of partners in the neighbouring slabs; the
//      neighbours' boundary rows;
//   3. expansion y_i = sum over the row's entries of (entry) (vector row it multiplies),
//      one table of vector rows per leaf, fixed for the whole launch;
//   4. the update of Algorithm 2.6.
// A CTA reads from exactly the CTAs that read from it (the interaction lists and the
// neighbour relation are symmetric), so no CTA runs two steps ahead of one that has not
// yet read its slot (the tags of sweep_team.cu).
#include <algorithm>
#include <cstdlib>
#include <vector>
#include "handle.h"
#include "sweep_common.cuh"
#include "tma.cuh"

namespace {

using namespace tma;
using namespace sweepc;

constexpr int kST = 512;                    // threads per CTA (one CTA per SM)
constexpr int kST2 = 256;                   // threads per CTA of the two-CTAs-per-SM variant
constexpr int kSKS = 8;                      // expansion: lanes per row
constexpr long long kSWait = 1LL << 22;      // bounded waits (about a second)

// offset of partner slot t of the cluster with index c at its depth
__host__ __device__ __forceinline__ int il_off(int c, int t) {
  return (c & 1) ? (t == 0 ? -3 : (t == 1 ? -2 : 2)) : (t == 0 ? -2 : (t == 1 ? 2 : 3));
}
// the slot of offset o in the list of the cluster with index c (-1 if none)
__host__ __device__ __forceinline__ int il_slot(int c, int o) {
  for (int t = 0; t < 3; ++t)
    if (il_off(c, t) == o) return t;
  return -1;
}

template <typename R>
struct StrongArgs {
  int n, L, leaf, dC, C, nteams, nrhs, ngroups, slab_max, nl, Rk, R3, ntask, nred_anc, nsub;
  long long N, layer_stride;
  unsigned stage_bytes;
  int xwords, aw, sw;           // exchange words per CTA and RHS: total, ancestors, subtree
  const int* lo;
  const int* sz;
  const long long* recoff;      // [nleaves + 1] record offsets within a layer (entries)
  const int* rstride;           // [nleaves]
  const Cx<R>* pack;
  const c128* north;
  const c128* r;
  c128* z;
  Cx<R>* w;
  typename Tagged<R>::W* xch;   // [2][nteams][C][xwords][G]
  int* status;
  long long wait_limit;
  int withhold;
  // shared-memory plan (byte offsets)
  unsigned o_stage[2], o_x[2], o_oq, o_qa, o_qr, o_zero, o_vt[2], o_vtoff, o_rrec, o_rrw, o_rleaf, o_task, o_lo,
      o_sz, o_mbar, o_flags;
};

// the setup's source of every strongly admissible entry, from the expanded factors:
//   src[(v * 3 + t) * 3 + {0,1,2}] = {node, first row of v in the node, column} of W_{v,t}
//   near[j * 3 + {0,1,2}] = {node, first row of leaf j in the node, column} of T(j, j + 1)
struct StrongSrc {
  const int* src;
  const int* nearr;
};

// One CTA per leaf: the records of layer m from the expanded factors G_F (node v at
// gfo[v], column-major, ld sz[v]) and the leaf blocks G_leaf (column-major, ld leaf).
template <typename R>
__global__ void strong_pack(int m, int L, int leaf, int R1, const int* __restrict__ lo, const int* __restrict__ sz,
                            const long long* __restrict__ gfo, StrongSrc ss, const Cx<R>* __restrict__ G_F,
                            const Cx<R>* __restrict__ G_leaf, const long long* __restrict__ recoff,
                            const int* __restrict__ rstride, Cx<R>* __restrict__ pack, long long layer_stride) {
  const int nleaves = 1 << L;
  const int j = blockIdx.x, lam = nleaves + j;
  const int s = sz[lam];
  const int sl = j > 0 ? sz[lam - 1] : 0, sr = j < nleaves - 1 ? sz[lam + 1] : 0;
  const int wb = s + sl + sr, R3 = 3 * R1, len = wb + R3 * (L - 1), rs = rstride[j];
  Cx<R>* out = pack + (long long)m * layer_stride + recoff[j];
  const long long tot = recoff[j + 1] - recoff[j];
  for (long long e0 = threadIdx.x; e0 < tot; e0 += blockDim.x) {
    const int i = (int)(e0 / rs), e = (int)(e0 % rs);
    Cx<R> v(0, 0);
    if (i < s && e < len) {
      if (e < s) {
        v = G_leaf[(long long)j * leaf * leaf + (long long)e * leaf + i];
      } else if (e < s + sl) {          // T(lam, lam - 1) = T(lam - 1, lam)^t
        const int* nr = ss.nearr + 3 * (j - 1);
        const int node = nr[0], r0 = nr[1], col = nr[2], c = e - s;
        v = G_F[gfo[node] + (long long)(col + i) * sz[node] + r0 + c];
      } else if (e < wb) {               // T(lam, lam + 1)
        const int* nr = ss.nearr + 3 * j;
        const int node = nr[0], r0 = nr[1], col = nr[2], c = e - s - sl;
        v = G_F[gfo[node] + (long long)(col + c) * sz[node] + r0 + i];
      } else {
        const int e2 = e - wb, d = 2 + e2 / R3, cc = e2 % R3, t = cc / R1, k = cc % R1;
        const int vd = lam >> (L - d);
        const int* sp = ss.src + ((long long)vd * 3 + t) * 3;
        if (sp[0] > 0) {
          const int node = sp[0], r0 = sp[1], col = sp[2], iv = lo[lam] - lo[vd] + i;
          v = G_F[gfo[node] + (long long)(col + k) * sz[node] + r0 + iv];
        }
      }
    }
    out[e0] = v;
  }
}

// NT threads per CTA: 512 with one CTA per SM, or 256 with two (the same registers per
// thread; one CTA's barrier waits are covered by the other's work)
template <typename R, int G, int NT>
__global__ void __launch_bounds__(NT, kST / NT) sweep_strong_kernel(StrongArgs<R> a) {
  extern __shared__ __align__(128) unsigned char sm[];
  using M = Mac<R>;
  using T = Tagged<R>;
  constexpr int GS = vstride<R>(G);
  const int tid = threadIdx.x, lane = tid & 31;
  const int n = a.n, L = a.L, dC = a.dC, nl = a.nl, lf = a.leaf, R1 = a.Rk, R3 = a.R3;
  const int team = blockIdx.x / a.C, c = blockIdx.x % a.C;
  const int vc = (1 << dC) + c;
  const int lam0 = vc << (L - dC);
  const int j0 = lam0 - (1 << L);            // first leaf index of the slab
  const int HL = lf;                          // halo rows before the slab in the x buffers
  Cx<R>* smc = reinterpret_cast<Cx<R>*>(sm);
  int* s_lo = reinterpret_cast<int*>(sm + a.o_lo);
  int* s_sz = reinterpret_cast<int*>(sm + a.o_sz);
  int* rrec = reinterpret_cast<int*>(sm + a.o_rrec);     // record offset of each slab row
  int* rrw = reinterpret_cast<int*>(sm + a.o_rrw);       // ... of its W entries
  int* rleaf = reinterpret_cast<int*>(sm + a.o_rleaf);
  int* vtoff = reinterpret_cast<int*>(sm + a.o_vtoff);
  int* task = reinterpret_cast<int*>(sm + a.o_task);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(sm + a.o_mbar);
  volatile int* s_fail = reinterpret_cast<volatile int*>(sm + a.o_flags);
  int* s_ctr = reinterpret_cast<int*>(sm + a.o_flags) + 1;
  Cx<R>* oq = reinterpret_cast<Cx<R>*>(sm + a.o_oq);     // [nsub][3R][GS] the slab's own clusters
  const int nnodes = 2 << L;

  for (int v = tid; v < nnodes; v += NT) { s_lo[v] = a.lo[v]; s_sz[v] = a.sz[v]; }
  for (int e = tid; e < GS; e += NT) reinterpret_cast<Cx<R>*>(sm + a.o_zero)[e] = Cx<R>(0, 0);
  if (tid == 0) {
    *s_fail = 0;
    s_ctr[0] = 0;
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int lo_c = s_lo[vc], ns = s_sz[vc];
  const long long rec0 = a.recoff[j0];
  // static tables: per row its record offset and leaf; per leaf its table offset
  for (int i = tid; i < ns; i += NT) {
    int v = vc;
    for (int d = dC; d < L; ++d) v = 2 * v + ((lo_c + i) >= s_lo[2 * v + 1] ? 1 : 0);
    const int jl = v - lam0, jj = j0 + jl;
    rleaf[i] = jl;
    rrec[i] = (int)(a.recoff[jj] - rec0) + (lo_c + i - s_lo[v]) * a.rstride[jj];
    rrw[i] = rrec[i] + s_sz[v] + (jj > 0 ? s_sz[v - 1] : 0) + (jj < (1 << L) - 1 ? s_sz[v + 1] : 0);
  }
  if (tid == 0) {
    int o = 0;
    for (int jl = 0; jl < nl; ++jl) {
      const int jj = j0 + jl, lam = lam0 + jl;
      const int s = s_sz[lam], sl = jj > 0 ? s_sz[lam - 1] : 0, sr = jj < (1 << L) - 1 ? s_sz[lam + 1] : 0;
      vtoff[jl] = o;
      o += s + sl + sr + R3 * (L - 1);
    }
    vtoff[nl] = o;
  }
  __syncthreads();
  // vector-row table per leaf and x parity (entry offsets from the base of shared memory)
  const int zero_off = (int)(a.o_zero / sizeof(Cx<R>));
  const int oq_off = (int)(a.o_oq / sizeof(Cx<R>)), qa_off = (int)(a.o_qa / sizeof(Cx<R>));
  const int qr_off = (int)(a.o_qr / sizeof(Cx<R>));
  for (int xp = 0; xp < 2; ++xp) {
    int* vt = reinterpret_cast<int*>(sm + a.o_vt[xp]);
    const int x_off = (int)(a.o_x[xp] / sizeof(Cx<R>));
    for (int e0 = tid; e0 < vtoff[nl]; e0 += NT) {
      int jl = 0;
      while (vtoff[jl + 1] <= e0) ++jl;
      const int e = e0 - vtoff[jl];
      const int jj = j0 + jl, lam = lam0 + jl;
      const int s = s_sz[lam], sl = jj > 0 ? s_sz[lam - 1] : 0, sr = jj < (1 << L) - 1 ? s_sz[lam + 1] : 0;
      const int ib = s_lo[lam] - lo_c, wb = s + sl + sr;
      int off;
      if (e < s) off = x_off + (HL + ib + e) * GS;
      else if (e < s + sl) off = x_off + (HL + ib - sl + (e - s)) * GS;
      else if (e < wb) off = x_off + (HL + ib + s + (e - s - sl)) * GS;
      else {
        const int e2 = e - wb, d = 2 + e2 / R3, cc = e2 % R3, t = cc / R1, k = cc % R1;
        const int vd = lam >> (L - d), vl = vd - (1 << d);
        const int pl = vl + il_off(vl, t);
        if (pl < 0 || pl >= (1 << d)) {
          off = zero_off;
        } else if (d <= dC) {
          off = qa_off + ((d - 2) * R3 + t * R1 + k) * GS;
        } else {
          const int owner = pl >> (d - dC);
          const int sbase = (1 << (d - dC)) - 2;            // clusters of shallower subtree depths
          if (owner == c) {
            const int tp = il_slot(pl, -il_off(vl, t));
            off = oq_off + ((sbase + pl - (c << (d - dC))) * R3 + tp * R1 + k) * GS;
          } else {
            off = qr_off + ((sbase + vl - (c << (d - dC))) * R3 + t * R1 + k) * GS;
          }
        }
      }
      vt[e0] = off;
    }
  }
  // gather tasks {dst (>= 0: entry offset; < 0: -1 - row offset in the current x buffer),
  // word, first source CTA, number of source CTAs}
  if (tid == 0) {
    int nt = 0;
    for (int d = 2; d <= dC; ++d) {
      const int al = c >> (dC - d);
      for (int t = 0; t < 3; ++t) {
        const int pl = al + il_off(al, t);
        if (pl < 0 || pl >= (1 << d)) continue;
        const int tp = il_slot(pl, -il_off(al, t));
        for (int k = 0; k < R1; ++k) {
          int* tk = task + 4 * nt++;
          tk[0] = qa_off + ((d - 2) * R3 + t * R1 + k) * GS;
          tk[1] = (d - 2) * R3 + tp * R1 + k;
          tk[2] = pl << (dC - d);
          tk[3] = 1 << (dC - d);
        }
      }
    }
    for (int d = dC + 1; d <= L; ++d) {
      const int sbase = (1 << (d - dC)) - 2;
      for (int vl = c << (d - dC); vl < (c + 1) << (d - dC); ++vl) {
        for (int t = 0; t < 3; ++t) {
          const int pl = vl + il_off(vl, t);
          if (pl < 0 || pl >= (1 << d)) continue;
          const int owner = pl >> (d - dC);
          if (owner == c) continue;
          const int tp = il_slot(pl, -il_off(vl, t));
          for (int k = 0; k < R1; ++k) {
            int* tk = task + 4 * nt++;
            tk[0] = qr_off + ((sbase + vl - (c << (d - dC))) * R3 + t * R1 + k) * GS;
            tk[1] = a.aw + (sbase + pl - (owner << (d - dC))) * R3 + tp * R1 + k;
            tk[2] = owner;
            tk[3] = 1;
          }
        }
      }
    }
    // neighbours' boundary rows: the left neighbour's last leaf, the right one's first
    if (c > 0) {
      const int sl = s_sz[lam0 - 1];
      for (int row = 0; row < sl; ++row) {
        int* tk = task + 4 * nt++;
        tk[0] = -1 - (HL - sl + row) * GS;
        tk[1] = a.aw + a.sw + lf + row;
        tk[2] = c - 1;
        tk[3] = 1;
      }
    }
    if (c < a.C - 1) {
      const int sr = s_sz[lam0 + nl];
      for (int row = 0; row < sr; ++row) {
        int* tk = task + 4 * nt++;
        tk[0] = -1 - (HL + ns + row) * GS;
        tk[1] = a.aw + a.sw + row;
        tk[2] = c + 1;
        tk[3] = 1;
      }
    }
    s_ctr[1] = nt;
  }
  __syncthreads();
  const int ntask = s_ctr[1];

  const int nsteps = 2 * n - 1;
  const int ngroups_team = a.ngroups > team ? (a.ngroups - 1 - team) / a.nteams + 1 : 0;
  const int total_steps = ngroups_team * nsteps;
  const unsigned rec_bytes = (unsigned)((a.recoff[j0 + nl] - rec0) * (long long)sizeof(Cx<R>));
  auto layer_of = [&](int s) { return s < n ? s : 2 * n - 2 - s; };
  auto produce = [&](int s, int slot) {
    if (tid != 0) return;
    const int m = layer_of(s);
    unsigned long long* mb = &mbar[slot];
    if (rec_bytes > a.stage_bytes || rec_bytes == 0) {
      if (rec_bytes > a.stage_bytes) report_error(a.status, HSWEEP_ERR_ARG, m);
      mbar_arrive(mb);
    } else {
      fence_proxy_async();
      mbar_expect_tx(mb, rec_bytes);
      bulk_g2s(sm + a.o_stage[slot], a.pack + (long long)m * a.layer_stride + rec0, rec_bytes, mb);
    }
  };
  if (total_steps > 0) produce(0, 0);
  int issued = total_steps > 0 ? 1 : 0;
  // reduction items: ancestors (d = 2..dC) first, then the slab's clusters by depth; each
  // item is (depth, cluster, chunk of 8 of the 3R columns)
  const int nch = (R3 + 7) / 8;
  const int n_anc = a.nred_anc * nch;
  const int n_items = n_anc + a.nsub * nch;

  int t = 0, s = 0, grp = team;
  for (; t < total_steps; ++t) {
    const int g0 = grp * G;
    const int gcount = (a.nrhs - g0) < G ? (a.nrhs - g0) : G;
    const bool fwd = s < n;
    const int m = fwd ? s : 2 * n - 2 - s;
    const int slot = t & 1;
    const unsigned tag = (unsigned)(t >> 1) & 1u;
    Cx<R>* xe = reinterpret_cast<Cx<R>*>(sm + a.o_x[s & 1]);           // row -HL at xe[0]
    Cx<R>* xne = reinterpret_cast<Cx<R>*>(sm + a.o_x[(s + 1) & 1]);
    Cx<R>* x = xe + HL * GS;
    Cx<R>* xn = xne + HL * GS;
    const int* vt = reinterpret_cast<const int*>(sm + a.o_vt[s & 1]);
    if (s == 0) {
      for (int it = tid; it < ns * G; it += NT) {
        const int i = it / G, g = it % G;
        Cx<R> v(0, 0);
        if (g < gcount) v = cvt<R>(a.r[(long long)(g0 + g) * a.N + lo_c + i]);
        x[i * GS + g] = v;
      }
      __syncthreads();
    }
    {   // the stage of step t (every thread observes the completed copy)
      long long spins = 0;
      while (!mbar_try_wait(&mbar[slot], (unsigned)((t >> 1) & 1))) {
        if (++spins > kSWait) {
          report_error(a.status, HSWEEP_ERR_TIMEOUT, m);
          *s_fail = 1;
          break;
        }
      }
    }
    const Cx<R>* st = reinterpret_cast<const Cx<R>*>(sm + a.o_stage[slot]);
    typename T::W* xpart = a.xch + (((long long)slot * a.nteams + team) * a.C + c) * a.xwords * G;
    const typename T::W* xteam = a.xch + ((long long)slot * a.nteams + team) * a.C * a.xwords * G;
    const bool pub = (int)blockIdx.x != a.withhold;

    // ---- 0. next bulk copy, L2 prefetch of the next update's inputs, boundary rows ----
    if (tid == 0 && t + 1 < total_steps) {
      produce(s + 1 == nsteps ? 0 : s + 1, slot ^ 1);
      issued = t + 2;
    }
    if (pub && a.C > 1) {
      const int sf = s_sz[lam0], sla = s_sz[lam0 + nl - 1];
      for (int it = tid; it < (sf + sla) * G; it += NT) {
        const int row = it / G, g = it % G;
        const int side = row < sf ? 0 : 1, rr = side ? row - sf : row;
        const int i = side ? ns - sla + rr : rr;
        T::store(xpart + (long long)(a.aw + a.sw + side * lf + rr) * G + g, T::pack(x[i * GS + g], tag));
      }
    }
    // ---- 1. reductions ------------------------------------------------------------------
    {
      const int kl = lane & 7, rl = lane >> 3;
      for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&s_ctr[0], 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        int d, rb, re, sidx = -1, ch;
        if (it < n_anc) {
          d = 2 + it / nch;
          ch = it % nch;
          rb = 0;
          re = ns;
        } else {
          const int it2 = (it - n_anc) / nch;
          ch = (it - n_anc) % nch;
          d = dC + 1;
          int base = 0;
          while (it2 >= base + (1 << (d - dC))) { base += 1 << (d - dC); ++d; }
          const int vl = it2 - base;
          const int v = (vc << (d - dC)) + vl;
          rb = s_lo[v] - lo_c;
          re = rb + s_sz[v];
          sidx = it2;
          if (d < 2) continue;              // depth 1 has no interaction list
        }
        const int cc = ch * 8 + kl;
        const bool lv = cc < R3;
        const int col = (d - 2) * R3 + (lv ? cc : 0);
        typename M::A acc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) M::zero(acc[g]);
#pragma unroll 4
        for (int i = rb + rl; i < re; i += 4) {
          const typename M::F f = M::f(st + rrw[i] + col);
          typename M::X xv[G];
          load_row<R, G>(x + i * GS, xv);
#pragma unroll
          for (int g = 0; g < G; ++g) M::mac(acc[g], f, xv[g]);
        }
        Cx<R> out[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          out[g] = M::get(acc[g]);
          out[g] += shfl_xor(out[g], 8);
          out[g] += shfl_xor(out[g], 16);
        }
        if (rl == 0 && lv) {
          if (sidx < 0) {
            if (pub)
#pragma unroll
              for (int g = 0; g < G; ++g) T::store(xpart + (long long)((d - 2) * R3 + cc) * G + g, T::pack(out[g], tag));
          } else {
#pragma unroll
            for (int g = 0; g < G; ++g) oq[(sidx * R3 + cc) * GS + g] = out[g];
            if (pub && a.C > 1)
#pragma unroll
              for (int g = 0; g < G; ++g) T::store(xpart + (long long)(a.aw + sidx * R3 + cc) * G + g, T::pack(out[g], tag));
          }
        }
      }
    }
    // ---- 2. gather --------------------------------------------------------------------
    for (int e = tid; e < ntask * G; e += NT) {
      const int k = e / G, g = e % G;
      const int* tk = task + 4 * k;
      const int nsrc = tk[3];
      const typename T::W* src = xteam + ((long long)tk[2] * a.xwords + tk[1]) * G + g;
      const long long cstride = (long long)a.xwords * G;
      Cx<R> acc(0, 0);
      for (int u0 = 0; u0 < nsrc; u0 += 8) {
        typename T::W vals[8];
        const int nu = min(8, nsrc - u0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (u < nu) vals[u] = T::load(src + (u0 + u) * cstride);
        long long spins = 0;
        for (;;) {
          bool pending = false;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (u < nu && !T::ok(vals[u], tag)) {
              vals[u] = T::load(src + (u0 + u) * cstride);
              pending = true;
            }
          if (!pending) break;
          if (++spins > a.wait_limit || *(volatile int*)a.status != 0) {
            report_error(a.status, HSWEEP_ERR_TIMEOUT, m);
            *s_fail = 1;
            break;
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (u < nu) acc += T::value(vals[u]);
      }
      const int dst = tk[0];
      if (dst >= 0) smc[dst + g] = acc;
      else xe[(-1 - dst) + g] = acc;
    }
    __syncthreads();
    if (*s_fail != 0) break;

    // ---- 3. expansion -----------------------------------------------------------------
    Cx<R>* ybuf = xn;
    for (int item = tid; item < ((ns * kSKS + 31) & ~31); item += NT) {
      const bool live = item < ns * kSKS;
      const int ks = item % kSKS;
      const int i = live ? item / kSKS : 0;
      const int jl = rleaf[i];
      const int e0 = vtoff[jl], len = vtoff[jl + 1] - e0;
      const Cx<R>* F = st + rrec[i];
      const int* vr = vt + e0;
      typename M::A acc[G];
#pragma unroll
      for (int g = 0; g < G; ++g) M::zero(acc[g]);
      if (live) {
        // not unrolled (measured: 14.5 against 15.1 ms per 64-RHS launch at n = 1023)
#pragma unroll 1
        for (int e = ks; e < len; e += kSKS) {
          const typename M::F f = M::f(F + e);
          typename M::X v[G];
          load_row<R, G>(smc + vr[e], v);
#pragma unroll
          for (int g = 0; g < G; ++g) M::mac(acc[g], f, v[g]);
        }
      }
      Cx<R> y[G];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        y[g] = M::get(acc[g]);
#pragma unroll
        for (int o = 1; o < kSKS; o <<= 1) y[g] += shfl_xor(y[g], o);
      }
      if (live && ks == 0) {
#pragma unroll
        for (int g = 0; g < G; ++g) ybuf[i * GS + g] = y[g];
      }
    }
    // the update's global inputs, issued before the barrier
    constexpr int kU = G >= 8 ? 1 : 2;
    c128 pcpl[kU], pin[kU];
    Cx<R> pw[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int p = tid + u * NT;
      pcpl[u] = c128(0.0, 0.0);
      pin[u] = c128(0.0, 0.0);
      pw[u] = Cx<R>(0, 0);
      if (p < ns * G) {
        const int i = p % ns, g = p / ns;
        const int mn = (fwd && m < n - 1) ? m + 1 : m;
        pcpl[u] = a.north[(long long)mn * n + lo_c + i];
        if (g < gcount) {
          if (fwd && m < n - 1) pin[u] = a.r[(long long)(g0 + g) * a.N + (long long)(m + 1) * n + lo_c + i];
          else if (!fwd) pw[u] = a.w[(long long)(g0 + g) * a.N + (long long)m * n + lo_c + i];
        }
      }
    }
    __syncthreads();
    // ---- 4. the update of Algorithm 2.6 ------------------------------------------------
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int p = tid + u * NT;
      if (p < ns * G) {
        const int i = p % ns, g = p / ns;
        const bool valid = g < gcount;
        const Cx<R> yv = ybuf[i * GS + g];
        const Cx<R> cpl = cvt<R>(pcpl[u]);
        const long long pos = (long long)(g0 + g) * a.N + (long long)m * n + lo_c + i;
        if (fwd) {
          if (m < n - 1) {
            if (valid) a.w[pos] = yv;
            xn[i * GS + g] = cvt<R>(pin[u]) - cpl * yv;
          } else {
            if (valid) a.z[pos] = cvt<double>(yv);
            xn[i * GS + g] = cpl * yv;
          }
        } else {
          const Cx<R> uu = valid ? pw[u] - yv : Cx<R>(0, 0);
          if (valid) a.z[pos] = cvt<double>(uu);
          if (m > 0) xn[i * GS + g] = cpl * uu;
        }
      }
    }
    if (tid == 0) s_ctr[0] = 0;
    __syncthreads();
    if (++s == nsteps) { s = 0; grp += a.nteams; }
  }
  // a CTA that stopped early still owns the bulk copies it issued: wait for them
  if (tid == 0) {
    for (int q = t + 1; q < issued; ++q) {
      long long spins = 0;
      const unsigned parity = (unsigned)((q >> 1) & 1);
      while (!mbar_try_wait(&mbar[q & 1], parity) && ++spins <= kSWait) {
      }
    }
  }
  __syncthreads();
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Host side: the static layout, the sources in the expanded factors, the records of a
// layer, the launch plan and the apply.

struct StrongPack {
  int R = 0;
  long long layer_stride = 0;            // entries per layer
  std::vector<long long> recoff;         // [nleaves + 1]
  std::vector<int> rstride;              // [nleaves]
  std::vector<long long> slab_bytes_max; // per slab depth dC (the same for every layer)
  long long* d_recoff = nullptr;
  int* d_rstride = nullptr;
  int* d_src = nullptr;
  int* d_near = nullptr;
  void* d_pack = nullptr;
  std::vector<std::array<long long, 9>> plans;   // {nrhs, ok, dC, C, G, teams, smem, ntask, threads}
};

namespace {

int depth_host(int v) { int d = 0; while (v > 1) { v >>= 1; ++d; } return d; }

// the sources of the strongly admissible entries in the expanded factors written by
// strong.cu (the same walk over sibling pairs and their corner chains)
void strong_sources(const Tree& t, int R, std::vector<int>& src, std::vector<int>& nearr) {
  const int L = t.L;
  src.assign((size_t)t.nnodes * 9, 0);
  nearr.assign((size_t)t.nleaves * 3, 0);
  for (int av = 2; av < t.nnodes; av += 2) {
    const int bv = av + 1, la = depth_host(av);
    int ca = av, cb = bv;
    for (int l = la + 1; l <= L; ++l) {
      const int us[3] = {2 * ca, 2 * ca, 2 * ca + 1};
      const int ws[3] = {2 * cb, 2 * cb + 1, 2 * cb + 1};
      for (int tt = 0; tt < 3; ++tt) {
        const int u = us[tt], w = ws[tt], col = R * (3 * (l - la - 1) + tt);
        const int ul = u - (1 << l), wl = w - (1 << l);
        const int tu = il_slot(ul, wl - ul), tw = il_slot(wl, ul - wl);
        int* su = &src[((size_t)u * 3 + tu) * 3];
        su[0] = av; su[1] = t.lo[u] - t.lo[av]; su[2] = col;
        int* sw = &src[((size_t)w * 3 + tw) * 3];
        sw[0] = bv; sw[1] = t.lo[w] - t.lo[bv]; sw[2] = col;
      }
      ca = 2 * ca + 1;
      cb = 2 * cb;
    }
    int* nr = &nearr[(size_t)(ca - t.nleaves) * 3];
    nr[0] = av; nr[1] = t.lo[ca] - t.lo[av]; nr[2] = 3 * R * (L - la);
  }
}

}  // namespace

void hsw_spack_free(hsweep_s* h) {
  if (!h->spk) return;
  StrongPack* p = h->spk;
  void* ptrs[] = {p->d_recoff, p->d_rstride, p->d_src, p->d_near, p->d_pack};
  for (void* q : ptrs) hsw_release(h, q);
  delete p;
  h->spk = nullptr;
  h->spack_valid = false;
}

static int spack_prepare(hsweep_s* h) {
  StrongPack* p = new (std::nothrow) StrongPack();
  if (!p) return HSWEEP_ERR_OOM;
  h->spk = p;
  const Tree& t = h->tree;
  const int R = h->strong_R, L = h->L;
  p->R = R;
  p->recoff.assign(t.nleaves + 1, 0);
  p->rstride.assign(t.nleaves, 0);
  for (int j = 0; j < t.nleaves; ++j) {
    const int lam = t.nleaves + j, s = t.sz[lam];
    const int sl = j > 0 ? t.sz[lam - 1] : 0, sr = j < t.nleaves - 1 ? t.sz[lam + 1] : 0;
    const int len = s + sl + sr + 3 * R * (L - 1);
    p->rstride[j] = len | 1;
    p->recoff[j + 1] = p->recoff[j] + (((long long)s * p->rstride[j] + 1) & ~1LL);
  }
  p->layer_stride = (p->recoff[t.nleaves] + 63) / 64 * 64;
  p->slab_bytes_max.assign(L + 1, 0);
  const size_t es = h->fac_elem();
  for (int dC = 0; dC <= L; ++dC) {
    const int nl = 1 << (L - dC);
    long long mx = 0;
    for (int cc = 0; cc < (1 << dC); ++cc) mx = std::max(mx, p->recoff[(cc + 1) * nl] - p->recoff[cc * nl]);
    p->slab_bytes_max[dC] = mx * (long long)es;
  }
  std::vector<int> src, nearr;
  strong_sources(t, R, src, nearr);
  int rc;
  if ((rc = hsw_alloc(h, (void**)&p->d_recoff, p->recoff.size() * sizeof(long long)))) return rc;
  if ((rc = hsw_alloc(h, (void**)&p->d_rstride, p->rstride.size() * sizeof(int)))) return rc;
  if ((rc = hsw_alloc(h, (void**)&p->d_src, src.size() * sizeof(int)))) return rc;
  if ((rc = hsw_alloc(h, (void**)&p->d_near, nearr.size() * sizeof(int)))) return rc;
  if ((rc = hsw_alloc(h, &p->d_pack, (size_t)h->n * p->layer_stride * es))) return rc;
  HSW_CUDA(cudaMemcpyAsync(p->d_recoff, p->recoff.data(), p->recoff.size() * sizeof(long long), cudaMemcpyHostToDevice,
                           h->stream));
  HSW_CUDA(cudaMemcpyAsync(p->d_rstride, p->rstride.data(), p->rstride.size() * sizeof(int), cudaMemcpyHostToDevice,
                           h->stream));
  HSW_CUDA(cudaMemcpyAsync(p->d_src, src.data(), src.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  HSW_CUDA(cudaMemcpyAsync(p->d_near, nearr.data(), nearr.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  HSW_CUDA(cudaStreamSynchronize(h->stream));   // the host vectors go out of scope
  return HSWEEP_OK;
}

int hsw_spack_layer(hsweep_s* h, int m, const void* G_F, const void* G_leaf, const long long* d_gfo) {
  if (h->strong_R <= 0) return HSWEEP_OK;
  if (!h->spk) {
    int rc = spack_prepare(h);
    if (rc) return rc;
  }
  StrongPack* p = h->spk;
  StrongSrc ss{p->d_src, p->d_near};
  if (h->prec == HSWEEP_FP64)
    strong_pack<double><<<h->nleaves, 128, 0, h->stream>>>(m, h->L, h->leaf, p->R, h->d_lo, h->d_sz, d_gfo, ss,
        (const c128*)G_F, (const c128*)G_leaf, p->d_recoff, p->d_rstride, (c128*)p->d_pack, p->layer_stride);
  else
    strong_pack<float><<<h->nleaves, 128, 0, h->stream>>>(m, h->L, h->leaf, p->R, h->d_lo, h->d_sz, d_gfo, ss,
        (const c64*)G_F, (const c64*)G_leaf, p->d_recoff, p->d_rstride, (c64*)p->d_pack, p->layer_stride);
  h->nlaunch += 1;
  HSW_CUDA(cudaGetLastError());
  if (m == h->n - 1) {
    h->spack_valid = true;
    p->plans.clear();
  }
  return HSWEEP_OK;
}

namespace {

struct StrongConfig {
  bool ok;
  int dC, C, G, nteams, ntask;
  size_t smem;
  int nt;              // threads per CTA (kST or kST2)
};

// shared-memory plan and exchange layout for (dC, G); 0 if not supported
template <typename R>
size_t plan_strong(const hsweep_s* h, int dC, int G, StrongArgs<R>& a, int nt = kST) {
  const StrongPack* p = h->spk;
  const size_t es = sizeof(Cx<R>);
  const int L = h->L, lf = h->leaf, R1 = p->R, R3 = 3 * R1;
  const int nl = 1 << (L - dC);
  const int slab_max = h->tree.maxsz(dC);
  const int GS = vstride<R>(G);
  if (L > 14 || L < 2 || (long long)slab_max * G > (G >= 8 ? 1LL : 2LL) * nt || lf > 8) return 0;
  auto al = [](size_t x, size_t b) { return (x + b - 1) / b * b; };
  const int nred_anc = dC >= 2 ? dC - 1 : 0;
  // the slab's own clusters are counted from depth dC + 1 (index base 2^(d - dC) - 2); a
  // depth-1 cluster (dC = 0) has no interaction list and its slots stay unused
  int nsub_slots = 0;
  for (int d = dC + 1; d <= L; ++d) nsub_slots += 1 << (d - dC);
  const int maxlen = 3 * lf + R3 * (L - 1);
  size_t o = 0;
  const size_t stage = al((size_t)p->slab_bytes_max[dC], 128);
  for (int b = 0; b < 2; ++b) { a.o_stage[b] = (unsigned)o; o += stage; }
  for (int b = 0; b < 2; ++b) { a.o_x[b] = (unsigned)o; o += al((size_t)(slab_max + 2 * lf) * GS * es, 16); }
  a.o_oq = (unsigned)o; o += al((size_t)std::max(1, nsub_slots) * R3 * GS * es, 16);
  a.o_qa = (unsigned)o; o += al((size_t)std::max(1, nred_anc) * R3 * GS * es, 16);
  a.o_qr = (unsigned)o; o += al((size_t)std::max(1, nsub_slots) * R3 * GS * es, 16);
  a.o_zero = (unsigned)o; o += al((size_t)GS * es, 16);
  for (int b = 0; b < 2; ++b) { a.o_vt[b] = (unsigned)o; o += al((size_t)nl * maxlen * sizeof(int), 16); }
  a.o_vtoff = (unsigned)o; o += al((size_t)(nl + 1) * sizeof(int), 16);
  a.o_rrec = (unsigned)o; o += al((size_t)slab_max * sizeof(int), 16);
  a.o_rrw = (unsigned)o; o += al((size_t)slab_max * sizeof(int), 16);
  a.o_rleaf = (unsigned)o; o += al((size_t)slab_max * sizeof(int), 16);
  const int ntask_max = nred_anc * R3 + nsub_slots * R3 + 2 * lf;
  a.o_task = (unsigned)o; o += al((size_t)std::max(1, ntask_max) * 4 * sizeof(int), 16);
  a.o_lo = (unsigned)o; o += al((size_t)h->nnodes * sizeof(int), 16);
  a.o_sz = (unsigned)o; o += al((size_t)h->nnodes * sizeof(int), 16);
  a.o_mbar = (unsigned)o; o += 16;
  a.o_flags = (unsigned)o; o += 16;
  a.stage_bytes = (unsigned)stage;
  a.nl = nl;
  a.slab_max = slab_max;
  a.Rk = R1;
  a.R3 = R3;
  a.nred_anc = nred_anc;
  a.nsub = nsub_slots;
  a.aw = nred_anc * R3;
  a.sw = nsub_slots * R3;
  a.xwords = a.aw + a.sw + 2 * lf;
  a.ntask = ntask_max;
  return o;
}

template <typename R, int G, int NT>
int resident_strong(const hsweep_s* h, size_t smem) {
  auto kern = sweep_strong_kernel<R, G, NT>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * h->num_sms;
}

template <typename R, int NT>
int resident_strong_g(const hsweep_s* h, int G, size_t smem) {
  switch (G) {
    case 1: return resident_strong<R, 1, NT>(h, smem);
    case 2: return resident_strong<R, 2, NT>(h, smem);
    case 4: return resident_strong<R, 4, NT>(h, smem);
    default: return resident_strong<R, 8, NT>(h, smem);
  }
}

// team size, right-hand sides per team and threads per CTA: the fewest rounds of 2n - 1
// steps, a step costing a fixed latency growing slowly with the team's size, work growing
// with the slab's rows times G, and a further latency for every extra pass of the expansion
// over the slab's rows (more than NT / kSKS rows per CTA of NT threads); coefficients from
// the measured apply at n = 1023 (64 RHS: teams of 16 CTAs with G = 8, 15.1 ms; 8 CTAs with
// G = 4, 16.2 ms; two CTAs of 256 threads per SM, 15.0-15.2 ms: no gain, so their work term
// is weighted up; one RHS: 32 CTAs 7.4 ms, 16 CTAs 8.1 ms)
// weight of the work term for two CTAs per SM (each CTA has half the threads)
constexpr double kShareS2 = 1.5;

template <typename R>
StrongConfig choose_strong(hsweep_s* h, int nrhs) {
  StrongPack* p = h->spk;
  for (const auto& e : p->plans)
    if (e[0] == nrhs)
      return StrongConfig{e[1] != 0, (int)e[2], (int)e[3], (int)e[4], (int)e[5], (int)e[7], (size_t)e[6], (int)e[8]};
  StrongConfig best{};
  best.ok = false;
  double best_cost = 1e300;
  const int C_pref = h->opt.team, G_pref = h->opt.groups, T_pref = h->opt.team_threads;
  for (int C = 1; C <= h->nleaves && C <= 2 * h->num_sms; C *= 2) {
    if (C_pref > 0 && C != C_pref) continue;
    int dC = 0;
    while ((1 << (dC + 1)) <= C) ++dC;
    for (int nt : {kST, kST2}) {
      if (T_pref > 0 && nt != T_pref) continue;
      for (int G : {8, 4, 2, 1}) {
        if (G_pref > 0 && G != G_pref) continue;
        StrongArgs<R> a;
        const size_t smem = plan_strong<R>(h, dC, G, a, nt);
        if (smem == 0 || smem > 227 * 1024) continue;
        const int resident = nt == kST2 ? resident_strong_g<R, kST2>(h, G, smem) : resident_strong_g<R, kST>(h, G, smem);
        const int teams_cap = std::min(resident, 1024) / C;
        if (teams_cap < 1) continue;
        if (nt == kST2 && resident < 2 * h->num_sms) continue;   // only where two CTAs fit per SM
        const int ngroups = (nrhs + G - 1) / G;
        const int teams = std::min(ngroups, teams_cap);
        const int rounds = (ngroups + teams - 1) / teams;
        const double es = (double)sizeof(Cx<R>) / 8.0;
        const int passes = (a.slab_max * kSKS + nt - 1) / nt;
        const double work = 0.006 * es * a.slab_max * G * ((double)kST / nt) * (nt == kST2 ? kShareS2 : 1.0);
        const double step = 2.5 + work + 0.005 * C + 1.0 * (passes - 1);
        const double cost = rounds * step;
        if (cost < best_cost - 1e-9) {
          best_cost = cost;
          best = StrongConfig{true, dC, C, G, teams, a.ntask, smem, nt};
        }
      }
    }
  }
  if (p->plans.size() >= 64) p->plans.erase(p->plans.begin());
  p->plans.push_back({nrhs, best.ok ? 1 : 0, best.dC, best.C, best.G, best.nteams, (long long)best.smem, best.ntask,
                      best.nt});
  return best;
}

long long al256s(long long x) { return (x + 255) / 256 * 256; }

template <typename R>
void strong_scratch_need(const hsweep_s* h, int nrhs, const StrongConfig& cfg, long long* w_bytes, long long* x_bytes) {
  StrongArgs<R> a;
  plan_strong<R>(h, cfg.dC, cfg.G, a, cfg.nt);
  const long long es = sizeof(Cx<R>);
  *w_bytes = (long long)nrhs * h->N * es;
  *x_bytes = 2LL * cfg.nteams * cfg.C * a.xwords * cfg.G * (long long)sizeof(typename Tagged<R>::W);
}

template <typename R, int G, int NT>
int launch_strong(hsweep_s* h, const StrongConfig& cfg, StrongArgs<R>& a) {
  auto kern = sweep_strong_kernel<R, G, NT>;
  HSW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem));
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[1];
  lc.blockDim = dim3(NT);
  lc.gridDim = dim3(cfg.C * cfg.nteams);
  lc.dynamicSmemBytes = cfg.smem;
  lc.stream = h->stream;
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->prof) {
    for (cudaEvent_t* e : {&e0, &e1}) {
      if (!h->ev_free.empty()) { *e = h->ev_free.back(); h->ev_free.pop_back(); }
      else HSW_CUDA(cudaEventCreate(e));
    }
    HSW_CUDA(cudaEventRecord(e0, h->stream));
  }
  HSW_CUDA(cudaLaunchKernelEx(&lc, kern, a));
  h->nlaunch += 1;
  if (h->prof) {
    HSW_CUDA(cudaEventRecord(e1, h->stream));
    h->ev_sweep.push_back({e0, e1});
  }
  return HSWEEP_OK;
}

template <typename R>
int apply_strong_impl(hsweep_s* h, const c128* r, c128* z, int nrhs, bool* used, void* scratch, size_t scratch_bytes) {
  *used = false;
  StrongConfig cfg = choose_strong<R>(h, nrhs);
  if (!cfg.ok) return HSWEEP_OK;
  const size_t es = sizeof(Cx<R>);
  long long wb, xb;
  strong_scratch_need<R>(h, nrhs, cfg, &wb, &xb);
  void *wptr, *xptr;
  if (scratch) {
    if ((size_t)(al256s(wb) + al256s(xb)) > scratch_bytes) return HSWEEP_ERR_ARG;
    wptr = scratch;
    xptr = (unsigned char*)scratch + al256s(wb);
  } else {
    const long long need_w = (long long)nrhs * h->N;
    if (need_w > h->wcache_cap) {
      int rc = hsw_regrow(h, &h->d_wcache, (size_t)need_w * es);
      if (rc) {
        if (!h->d_wcache) h->wcache_cap = 0;
        return rc;
      }
      h->wcache_cap = need_w;
    }
    const long long need_x = (xb + (long long)es - 1) / (long long)es;
    if (need_x > h->xch_cap) {
      int rc = hsw_regrow(h, &h->d_xch, (size_t)need_x * es);
      if (rc) {
        if (!h->d_xch) h->xch_cap = 0;
        return rc;
      }
      h->xch_cap = need_x;
    }
    wptr = h->d_wcache;
    xptr = h->d_xch;
  }
  StrongPack* p = h->spk;
  StrongArgs<R> a;
  plan_strong<R>(h, cfg.dC, cfg.G, a, cfg.nt);
  a.n = h->n; a.L = h->L; a.leaf = h->leaf; a.dC = cfg.dC; a.C = cfg.C; a.nteams = cfg.nteams; a.nrhs = nrhs;
  a.ngroups = (nrhs + cfg.G - 1) / cfg.G;
  a.N = h->N; a.layer_stride = p->layer_stride;
  a.lo = h->d_lo; a.sz = h->d_sz; a.recoff = p->d_recoff; a.rstride = p->d_rstride;
  a.pack = reinterpret_cast<const Cx<R>*>(p->d_pack);
  a.north = h->d_north_m; a.r = r; a.z = z;
  a.w = reinterpret_cast<Cx<R>*>(wptr);
  a.xch = reinterpret_cast<typename Tagged<R>::W*>(xptr);
  a.status = h->d_status;
  a.wait_limit = kSWait;
  a.withhold = -1;
  if (const char* e = getenv("HSWEEP_TEST_WAIT_LIMIT")) {
    const long long v = atoll(e);
    if (v > 0 && v < kSWait) a.wait_limit = v;
  }
  if (const char* e = getenv("HSWEEP_TEST_WITHHOLD")) a.withhold = atoi(e);
  const bool prof = h->prof;
  if (scratch) h->prof = false;
  int rc = HSWEEP_OK;
  // every exchange slot starts with the tag bit set: steps 0 and 1 expect it clear
  if (cudaMemsetAsync(xptr, 0xff, (size_t)xb, h->stream) != cudaSuccess) rc = HSWEEP_ERR_CUDA;
  if (rc == HSWEEP_OK) {
    if (cfg.nt == kST2) {
      switch (cfg.G) {
        case 1: rc = launch_strong<R, 1, kST2>(h, cfg, a); break;
        case 2: rc = launch_strong<R, 2, kST2>(h, cfg, a); break;
        case 4: rc = launch_strong<R, 4, kST2>(h, cfg, a); break;
        default: rc = launch_strong<R, 8, kST2>(h, cfg, a); break;
      }
    } else {
      switch (cfg.G) {
        case 1: rc = launch_strong<R, 1, kST>(h, cfg, a); break;
        case 2: rc = launch_strong<R, 2, kST>(h, cfg, a); break;
        case 4: rc = launch_strong<R, 4, kST>(h, cfg, a); break;
        default: rc = launch_strong<R, 8, kST>(h, cfg, a); break;
      }
    }
  }
  h->prof = prof;
  if (rc == HSWEEP_OK) *used = true;
  return rc;
}

}  // namespace

int hsw_apply_strong(hsweep_s* h, const c128* r, c128* z, int nrhs, bool* used, void* scratch, size_t scratch_bytes) {
  *used = false;
  if (!h->spack_valid || !h->spk) return HSWEEP_OK;
  if (h->prec == HSWEEP_FP64) return apply_strong_impl<double>(h, r, z, nrhs, used, scratch, scratch_bytes);
  return apply_strong_impl<float>(h, r, z, nrhs, used, scratch, scratch_bytes);
}

size_t hsw_apply_strong_scratch_bytes(hsweep_s* h, int nrhs) {
  if (!h->spack_valid || !h->spk) return 0;
  long long wb, xb;
  if (h->prec == HSWEEP_FP64) {
    StrongConfig cfg = choose_strong<double>(h, nrhs);
    if (!cfg.ok) return 0;
    strong_scratch_need<double>(h, nrhs, cfg, &wb, &xb);
  } else {
    StrongConfig cfg = choose_strong<float>(h, nrhs);
    if (!cfg.ok) return 0;
    strong_scratch_need<float>(h, nrhs, cfg, &wb, &xb);
  }
  return (size_t)(al256s(wb) + al256s(xb));
}

int hsw_strong_plan_sweep(hsweep_s* h, int nrhs, long long* out) {
  if (!h->spack_valid || !h->spk) return 0;
  StrongConfig cfg = h->prec == HSWEEP_FP64 ? choose_strong<double>(h, nrhs) : choose_strong<float>(h, nrhs);
  if (!cfg.ok) return 0;
  out[0] = 3; out[1] = cfg.C; out[2] = cfg.G; out[3] = cfg.nteams; out[4] = cfg.nt;
  out[5] = (long long)cfg.smem; out[6] = h->spk->slab_bytes_max[cfg.dC]; out[7] = kSKS;
  return 1;
}

extern "C" int hsweep_strong_export(hsweep_t h, int m, hsw_c128* records, long long* recoff, int* rstride,
                                    long long* nentries) {
  if (!h || !h->spack_valid || !h->spk || m < 0 || m >= h->n) return HSWEEP_ERR_ARG;
  StrongPack* p = h->spk;
  const long long ne = p->recoff[h->nleaves];
  if (nentries) *nentries = ne;
  if (recoff) std::copy(p->recoff.begin(), p->recoff.end(), recoff);
  if (rstride) std::copy(p->rstride.begin(), p->rstride.end(), rstride);
  if (records) {
    const size_t es = h->fac_elem();
    std::vector<unsigned char> buf((size_t)ne * es);
    HSW_CUDA(cudaStreamSynchronize(h->stream));
    HSW_CUDA(cudaMemcpy(buf.data(), (const unsigned char*)p->d_pack + (size_t)m * p->layer_stride * es, buf.size(),
                        cudaMemcpyDeviceToHost));
    for (long long i = 0; i < ne; ++i) {
      if (es == sizeof(c128)) {
        const c128 v = reinterpret_cast<const c128*>(buf.data())[i];
        records[i].re = v.re; records[i].im = v.im;
      } else {
        const c64 v = reinterpret_cast<const c64*>(buf.data())[i];
        records[i].re = v.re; records[i].im = v.im;
      }
    }
  }
  return HSWEEP_OK;
}
