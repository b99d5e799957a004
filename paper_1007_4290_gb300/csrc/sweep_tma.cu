// The apply z = M r of Algorithm 2.6 with the factors streamed by TMA.
//
// Same team organisation as the basic sweep kernel (apply.cu): a team of C = 2^dC CTAs
// carries G right-hand sides through the 2n-1 dependent hmatvecs; CTA c owns the rows
// of the depth-dC tree node vc = 2^dC + c.  What changes is how the factors arrive:
//   - the factors of a layer restricted to a CTA's rows are one contiguous record of
//     the leaf-major packed layout (pack.cu); one cp.async.bulk copy per step brings it
//     into shared memory, completing on an mbarrier;
//   - two stages: while step s computes from stage s&1, the copy for step s+1 (a layer
//     that does not depend on u) is already in flight, so the HBM stream is decoupled
//     from the chain of dependent layers;
//   - all arithmetic reads shared memory: reductions q_v = F_v^t x with lanes over the
//     columns k (contiguous in a row-major row), expansions y_i = sum_k F_v[i, k] q[k]
//     with lanes over rows (odd row strides: no bank conflicts), four right-hand sides
//     per thread from vector broadcast loads;
//   - the ancestors' partial sums are exchanged through L2 (st.cg / ld.cg), ordered by
//     one hardware cluster barrier per step when the team is a thread-block cluster, or
//     by a bounded-spin grid barrier when the team is the whole grid.
// (The default apply uses sweep_team.cu; this kernel is selected by sweep_kernel = 2 or
// when the cooperative-team plan does not fit.)
#include <cooperative_groups.h>
#include "handle.h"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace {

using namespace tma;

constexpr int kThreads = 512;
constexpr long long kWaitLimit = 1LL << 22;      // bounded waits (about a second)

template <typename R>
struct TmaArgs {
  int n, L, leaf, nnodes, dC, C, nteams, nrhs, ngroups, slab_max, nl, rcap, KS;
  long long N, pack_stride;
  unsigned stage_bytes;
  const int* lo;
  const int* sz;
  const int* rank;
  const long long* recoff;
  const Cx<R>* pack;
  const c128* north;
  const c128* r;
  c128* z;
  Cx<R>* w;
  Cx<R>* xch;        // ancestors' partial sums: [2][nteams][C][dC][rcap][G]
  int* status;
  unsigned* bar;
  // shared-memory plan (byte offsets)
  unsigned o_stage[2], o_rowoff[2], o_trk[3], o_ro[3], o_vin[2], o_vn[2], o_lo, o_sz, o_leafnode, o_dtab, o_wdesc, o_boff, o_x[2],
      o_qanc, o_qloc, o_mbar, o_flags;
};

// Bounded-spin barrier over the whole cooperative grid (see apply.cu).
__device__ bool grid_barrier2(unsigned* bar, unsigned nblocks, int* status, int layer) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = bar + 1;
    unsigned gen = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*vgen == gen) {
        if (++spins > kWaitLimit) { ok = 0; report_error(status, HSWEEP_ERR_TIMEOUT, layer); break; }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int*)status != 0) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// per-depth table columns in shared memory (16 ints each)
enum { DT_KW = 0, DT_NODES = 16, DT_QCAP = 32, DT_WSTART = 48, DT_QBASE = 64, DT_SIZE = 80 };

template <typename R, int G, bool GRID>
__global__ void __launch_bounds__(kThreads, 1) sweep_tma_kernel(TmaArgs<R> a) {
  extern __shared__ __align__(128) unsigned char sm[];
  constexpr int GC = G <= 5 ? G : 4;    // right-hand sides per thread
  constexpr int GQ = G / GC;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // arithmetic threads are warps 1..; warp 0 (the producer) starts every arithmetic loop
  // beyond its end, so it skips them
  const int ctid = tid >= 32 ? tid - 32 : (1 << 30), cnt = (int)blockDim.x - 32;
  const int cw = warp >= 1 ? warp - 1 : (1 << 30), ncw = (int)(blockDim.x >> 5) - 1;
  const int n = a.n, L = a.L, dC = a.dC, nl = a.nl, lf = a.leaf, SM = a.slab_max;
  const int c = GRID ? blockIdx.x : (int)cg::this_cluster().block_rank();
  const int team = GRID ? 0 : blockIdx.x / a.C;
  const int vc = (1 << dC) + c;
  const int lam0 = vc << (L - dC);          // first leaf node of the slab
  const int jglob0 = lam0 - (1 << L);       // its leaf index

  int* s_lo = reinterpret_cast<int*>(sm + a.o_lo);
  int* s_sz = reinterpret_cast<int*>(sm + a.o_sz);
  int* s_leafnode = reinterpret_cast<int*>(sm + a.o_leafnode);
  int* dt = reinterpret_cast<int*>(sm + a.o_dtab);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(sm + a.o_mbar);
  int* s_flags = reinterpret_cast<int*>(sm + a.o_flags);    // [0]: this CTA failed
  Cx<R>* qanc = reinterpret_cast<Cx<R>*>(sm + a.o_qanc);
  Cx<R>* qloc = reinterpret_cast<Cx<R>*>(sm + a.o_qloc);

  for (int v = tid; v < a.nnodes; v += blockDim.x) { s_lo[v] = a.lo[v]; s_sz[v] = a.sz[v]; }
  __syncthreads();
  const int lo_c = s_lo[vc], ns = s_sz[vc];
  if (tid == 0) {
    // reduction work per depth: a warp-item is (node, chunk of KW columns, block of GC
    // right-hand sides); its lanes are KW columns x (32 / KW) interleaved row subsets
    int wsum = 0, qb = 0;
    for (int d = 1; d <= L; ++d) {
      const int rows = d <= dC ? ns : (n + (1 << d) - 1) >> d;
      const int nodes = d <= dC ? 1 : (1 << (d - dC));
      const int qcap = d <= dC ? a.rcap : min(rows, a.rcap);
      int kw = 1;
      const int kwmax = d <= dC ? 8 : 16;
      while (kw < qcap && kw < kwmax) kw <<= 1;
      dt[DT_KW + d] = kw;
      dt[DT_NODES + d] = nodes;
      dt[DT_QCAP + d] = qcap;
      dt[DT_WSTART + d] = wsum;
      wsum += nodes * ((qcap + kw - 1) / kw) * GQ;
      dt[DT_QBASE + d] = qb;
      if (d > dC) qb += nodes * qcap * G;
    }
    // descriptors of every reduction warp-item: d | kc << 4 | jn << 12 | gq << 24
    {
      int* wdesc = reinterpret_cast<int*>(sm + a.o_wdesc);
      int wi = 0;
      for (int d = 1; d <= L; ++d) {
        const int nodes = dt[DT_NODES + d], qcap = dt[DT_QCAP + d], kw = dt[DT_KW + d];
        const int nkc = (qcap + kw - 1) / kw;
        for (int gq = 0; gq < GQ; ++gq)
          for (int jn = 0; jn < nodes; ++jn)
            for (int kc = 0; kc < nkc; ++kc) wdesc[wi++] = d | (kc << 4) | (jn << 12) | (gq << 24);
      }
    }
    dt[DT_WSTART + L + 1] = wsum;
    s_flags[0] = 0;
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  for (int i = tid; i < ns; i += blockDim.x) {
    int v = vc;
    for (int d = dC; d < L; ++d) v = 2 * v + ((lo_c + i) >= s_lo[2 * v + 1] ? 1 : 0);
    s_leafnode[i] = v;
  }
  __syncthreads();

  const int nsteps = 2 * n - 1;
  const int ngroups_team = a.ngroups > team ? (a.ngroups - 1 - team) / a.nteams + 1 : 0;
  const long long total_steps = (long long)ngroups_team * nsteps;

  // ---- producer (warp 0): everything step t needs that does not depend on u ----------
  //   load_tables(t): cp.async of the ranks of the slab's nodes and the record offsets of
  //     step t (issued two steps ahead, slot t % 3);
  //   produce(t): the per-row offsets of every block in the stage, one bulk copy of the
  //     factor record (mbarrier), and cp.async copies of the vectors the step's update
  //     reads (f_{m+1} or w_m, and the coupling), one step ahead.
  auto step_layer = [&](long long t) {
    const int s = (int)(t % nsteps);
    return s < n ? s : 2 * n - 2 - s;
  };
  auto load_tables = [&](long long t) {
    if (warp != 0 || t >= total_steps) return;
    const int m = step_layer(t);
    const int slot3 = (int)(t % 3);
    int* trk = reinterpret_cast<int*>(sm + a.o_trk[slot3]);
    long long* sro = reinterpret_cast<long long*>(sm + a.o_ro[slot3]);
    const int* rk = a.rank + (long long)m * a.nnodes;
    const long long* ro = a.recoff + (long long)m * ((long long)(1 << L) + 1);
    const int nloc = 2 * nl - 2;
    for (int q = lane; q < dC + nloc + nl + 1; q += 32) {
      if (q < dC) {
        cp_async4(trk + q, rk + (vc >> (dC - 1 - q)));
      } else if (q < dC + nloc) {
        const int li = q - dC;
        int dd = 1;
        while ((1 << (dd + 1)) - 2 <= li) ++dd;
        cp_async4(trk + q, rk + (vc << dd) + (li - ((1 << dd) - 2)));
      } else {
        const int j = q - dC - nloc;
        cp_async8(sro + j, ro + jglob0 + j);
      }
    }
  };
  // per-row offsets of every block of step t's record (from the tables in slot t % 3),
  // computed by one warp: first the block offsets and row strides of every slab leaf
  // (one lane per leaf), then one multiply-add per (row, depth)
  auto build_rowoff = [&](long long t) {
    if (t >= total_steps) return;
    int* rowoff = reinterpret_cast<int*>(sm + a.o_rowoff[t & 1]);
    const int* trk = reinterpret_cast<const int*>(sm + a.o_trk[t % 3]);
    const long long* sro = reinterpret_cast<const long long*>(sm + a.o_ro[t % 3]);
    int* boff = reinterpret_cast<int*>(sm + a.o_boff);          // [nl][L+1]
    int* brs = boff + nl * (L + 1);                             // [nl][L+1]
    for (int j = lane; j < nl; j += 32) {
      const int lam = lam0 + j;
      const int sl = s_sz[lam];
      int o = (int)(sro[j] - sro[0]);
      boff[j * (L + 1)] = o;
      brs[j * (L + 1)] = lf;
      o += lf * lf;
      for (int d = 1; d <= L; ++d) {
        int r;
        if (d <= dC) r = trk[d - 1];
        else {
          const int q = d - dC;
          r = trk[dC + (1 << q) - 2 + ((lam >> (L - d)) - (vc << q))];
        }
        const int rs = row_stride(r);
        boff[j * (L + 1) + d] = o;
        brs[j * (L + 1) + d] = rs;
        o += sl * rs;
      }
    }
    __syncwarp();
    for (int e = lane; e < ns * (L + 1); e += 32) {
      const int i = e % ns, d = e / ns;
      const int lam = s_leafnode[i];
      const int j = lam - lam0;
      const int ai = lo_c + i - s_lo[lam];
      rowoff[d * SM + i] = boff[j * (L + 1) + d] + ai * brs[j * (L + 1) + d];
    }
    __syncwarp();
  };
  // warp 0: the bulk copy of step t's factor record and cp.async of its update vectors
  auto produce = [&](long long t) {
    if (warp != 0 || t >= total_steps) return;
    const int s = (int)(t % nsteps);
    const int m = step_layer(t);
    const int slot = (int)(t & 1);
    const long long* sro = reinterpret_cast<const long long*>(sm + a.o_ro[t % 3]);
    {
      const int grp = team + (int)(t / nsteps) * a.nteams;
      const int g0 = grp * G;
      const int gcnt = (a.nrhs - g0) < G ? (a.nrhs - g0) : G;
      const bool fwd = s < n;
      unsigned char* vin = sm + a.o_vin[slot];
      c128* vn = reinterpret_cast<c128*>(sm + a.o_vn[slot]);
      const int mn = (fwd && m < n - 1) ? m + 1 : m;
      for (int i = lane; i < ns; i += 32) cp_async16(vn + i, a.north + (long long)mn * n + lo_c + i);
      if (fwd && m < n - 1) {
        c128* vr = reinterpret_cast<c128*>(vin);
        for (int e = lane; e < gcnt * ns; e += 32) {
          const int g = e / ns, i = e % ns;
          cp_async16(vr + g * SM + i, a.r + (long long)(g0 + g) * a.N + (long long)(m + 1) * n + lo_c + i);
        }
      } else if (!fwd) {
        Cx<R>* vw = reinterpret_cast<Cx<R>*>(vin);
        for (int e = lane; e < gcnt * ns; e += 32) {
          const int g = e / ns, i = e % ns;
          const Cx<R>* src = a.w + (long long)(g0 + g) * a.N + (long long)m * n + lo_c + i;
          if (sizeof(Cx<R>) == 16) cp_async16(vw + g * SM + i, src);
          else cp_async8(vw + g * SM + i, src);
        }
      }
    }
    if (lane == 0) {
      unsigned bytes = (unsigned)((sro[nl] - sro[0]) * (long long)sizeof(Cx<R>));
      unsigned long long* mb = &mbar[slot];
      if (bytes > a.stage_bytes || bytes == 0) {
        if (bytes > a.stage_bytes) report_error(a.status, HSWEEP_ERR_ARG, m);
        mbar_arrive(mb);      // complete the phase without data
      } else {
        fence_proxy_async();
        mbar_expect_tx(mb, bytes);
        bulk_g2s(sm + a.o_stage[slot], a.pack + (long long)m * a.pack_stride + sro[0], bytes, mb);
      }
    }
  };

  if (warp == 0) {
    load_tables(0);
    load_tables(1);
    cp_async_commit();
    cp_async_wait0();
    __syncwarp();
    produce(0);          // its vectors complete with the first wait of step 0
    cp_async_commit();
  }
  if (warp == 0) build_rowoff(0);
  __syncthreads();
  long long t = 0;
  for (int grp = team; grp < a.ngroups; grp += a.nteams) {
    const int g0 = grp * G;
    const int gcount = (a.nrhs - g0) < G ? (a.nrhs - g0) : G;
    {
      Cx<R>* x0 = reinterpret_cast<Cx<R>*>(sm + a.o_x[0]);
      for (int it = ctid; it < ns * G; it += cnt) {
        const int i = it / G, g = it % G;
        Cx<R> v(0, 0);
        if (g < gcount) v = cvt<R>(a.r[(long long)(g0 + g) * a.N + lo_c + i]);
        x0[i * G + g] = v;
      }
    }
    __syncthreads();
    for (int s = 0; s < nsteps; ++s, ++t) {
      const bool fwd = s < n;
      const int m = fwd ? s : 2 * n - 2 - s;
      const int slot = (int)(t & 1);
      const int par = s & 1;
      Cx<R>* x = reinterpret_cast<Cx<R>*>(sm + a.o_x[s & 1]);
      Cx<R>* xn = reinterpret_cast<Cx<R>*>(sm + a.o_x[(s + 1) & 1]);
      if (warp == 0) {
        cp_async_wait0();      // the vectors of step t and the tables of step t+1
        __syncwarp();
        produce(t + 1);
        load_tables(t + 2);
        cp_async_commit();
        // the next step's per-row offsets, while the other warps reduce
        build_rowoff(t + 1);
      }
      {
        long long spins = 0;
        const unsigned parity = (unsigned)((t >> 1) & 1);
        while (!mbar_try_wait(&mbar[slot], parity)) {
          if (++spins > kWaitLimit) {
            if (tid == 0) report_error(a.status, HSWEEP_ERR_TIMEOUT, m);
            s_flags[0] = 1;
            break;
          }
        }
      }
      const Cx<R>* st = reinterpret_cast<const Cx<R>*>(sm + a.o_stage[slot]);
      const int* rowoff = reinterpret_cast<const int*>(sm + a.o_rowoff[slot]);
      const int* trk = reinterpret_cast<const int*>(sm + a.o_trk[t % 3]);
      // no block barrier here: every thread waited on the stage's mbarrier itself; the
      // step's other inputs were completed before the previous step's last barrier, and
      // the update's vectors are ordered by the barrier after the gather
      const bool ok = s_flags[0] == 0;

      // ---- 1. reductions q_v[k][g] = sum_i F_v[i, k] x[i][g] ---------------------------
      //   warp-item (node, KW columns, GC right-hand sides): lane = (column kl, row set rl);
      //   each lane sums every (32/KW)-th row of the node, then the row sets are combined
      //   with log2(32/KW) shuffles.
      if (ok) {
        const int wtot = dt[DT_WSTART + L + 1];
        const int* wdesc = reinterpret_cast<const int*>(sm + a.o_wdesc);
        for (int wi = cw; wi < wtot; wi += ncw) {
          const int desc = wdesc[wi];
          const int d = desc & 15, kc = (desc >> 4) & 255, jn = (desc >> 12) & 4095, gq = desc >> 24;
          const int kw = dt[DT_KW + d], nodes = dt[DT_NODES + d], qcap = dt[DT_QCAP + d];
          const int kl = lane % kw, rl = lane / kw, rw = 32 / kw;
          const int k = kc * kw + kl;
          int r, rb, re;
          if (d <= dC) {
            r = trk[d - 1];
            rb = 0;
            re = ns;
          } else {
            const int v = (vc << (d - dC)) + jn;
            r = trk[dC + nodes - 2 + jn];
            rb = s_lo[v] - lo_c;
            re = rb + s_sz[v];
          }
          Cx<R> acc[GC];
#pragma unroll
          for (int g = 0; g < GC; ++g) acc[g] = Cx<R>(0, 0);
          if (k < r) {
            const int* ro_d = rowoff + d * SM;
            const Cx<R>* xq = x + gq * GC;
#pragma unroll 4
            for (int i = rb + rl; i < re; i += rw) {
              const Cx<R> f = st[ro_d[i] + k];
              const Cx<R>* xr = xq + i * G;
#pragma unroll
              for (int g = 0; g < GC; ++g) cfma(acc[g], f, xr[g]);
            }
          }
#pragma unroll
          for (int g = 0; g < GC; ++g)
            for (int o = kw; o < 32; o <<= 1) acc[g] += shfl_xor(acc[g], o);
          if (rl == 0 && k < qcap) {
            if (d <= dC) {
              Cx<R>* dst = a.xch +
                           ((((long long)par * a.nteams + team) * a.C + c) * dC + (d - 1)) * a.rcap * G + k * G + gq * GC;
#pragma unroll
              for (int g = 0; g < GC; ++g) st_cg(dst + g, acc[g]);
            } else {
              Cx<R>* dst = qloc + dt[DT_QBASE + d] + (jn * qcap + k) * G + gq * GC;
#pragma unroll
              for (int g = 0; g < GC; ++g) dst[g] = acc[g];
            }
          }
        }
      }

      // ---- 2. team barrier and the ancestors' sibling sums -------------------------
      bool alive = true;
      if (GRID) {
        alive = grid_barrier2(a.bar, gridDim.x, a.status, m);
      } else {
        cg::this_cluster().sync();
      }
      if (ok && alive) {
        for (int it = ctid; it < dC * a.rcap * G; it += cnt) {
          const int d = it / (a.rcap * G) + 1;
          const int kg = it - (d - 1) * a.rcap * G;
          const int v = vc >> (dC - d);
          const int span = 1 << (dC - d);
          const int c0 = ((v ^ 1) << (dC - d)) - (1 << dC);
          Cx<R> acc(0, 0);
          if (kg / G < trk[d - 1]) {
            const Cx<R>* src = a.xch + (((long long)par * a.nteams + team) * a.C * dC + (d - 1)) * a.rcap * G + kg;
            const long long cstride = (long long)dC * a.rcap * G;
            for (int cc = 0; cc < span; cc += 8) {
              Cx<R> vals[8];
#pragma unroll
              for (int u = 0; u < 8; ++u)
                vals[u] = (cc + u < span) ? ld_cg(src + (long long)(c0 + cc + u) * cstride) : Cx<R>(0, 0);
#pragma unroll
              for (int u = 0; u < 8; ++u) acc += vals[u];
            }
          }
          qanc[it] = acc;
        }
      }
      __syncthreads();

      // ---- 3. expansion y_i = D x + sum_v F_v[i, :] q_sib(v), and the sweep update ----
      //   item (row i, RHS block gq, column slice ks): the KS slices of a row are adjacent
      //   lanes of one warp and are summed by shuffles; the lane of slice 0 then applies
      //   the update of Algorithm 2.6 for its row.  Meanwhile the next step's per-row
      //   offsets are built by the same threads.
      if (ok && alive) {
        const int KS = a.KS;
        const unsigned char* vin = sm + a.o_vin[slot];
        const c128* vn = reinterpret_cast<const c128*>(sm + a.o_vn[slot]);
        const int nitems = ns * GQ * KS;
        const int nitems_r = (nitems + 31) & ~31;     // whole warps, so the shuffles are converged
        for (int item = tid; item < nitems_r; item += blockDim.x) {
          const bool live = item < nitems;
          const int ks = item % KS;
          const int rest = item / KS;
          const int i = live ? rest % ns : 0, gq = live ? rest / ns : 0;
          const int lam = s_leafnode[i];
          Cx<R> acc[GC];
#pragma unroll
          for (int g = 0; g < GC; ++g) acc[g] = Cx<R>(0, 0);
          if (live) {
            {
              const Cx<R>* D = st + rowoff[i];
              const Cx<R>* xb = x + (s_lo[lam] - lo_c) * G + gq * GC;
              const int sl = s_sz[lam];
              for (int b = ks; b < sl; b += KS) {
                const Cx<R> f = D[b];
#pragma unroll
                for (int g = 0; g < GC; ++g) cfma(acc[g], f, xb[b * G + g]);
              }
            }
            for (int d = 1; d <= L; ++d) {
              const Cx<R>* q;
              int r;
              if (d <= dC) {
                r = trk[d - 1];
                q = qanc + (d - 1) * a.rcap * G;
              } else {
                const int nodes = 1 << (d - dC);
                const int jn = (lam >> (L - d)) - (vc << (d - dC));
                r = trk[dC + nodes - 2 + jn];
                q = qloc + dt[DT_QBASE + d] + ((jn ^ 1) * dt[DT_QCAP + d]) * G;
              }
              const Cx<R>* Fr = st + rowoff[d * SM + i];
              const Cx<R>* qg = q + gq * GC;
#pragma unroll 4
              for (int k = ks; k < r; k += KS) {
                const Cx<R> f = Fr[k];
                const Cx<R>* qk = qg + k * G;
#pragma unroll
                for (int g = 0; g < GC; ++g) cfma(acc[g], f, qk[g]);
              }
            }
          }
#pragma unroll
          for (int g = 0; g < GC; ++g)
            for (int o = 1; o < KS; o <<= 1) acc[g] += shfl_xor(acc[g], o);
          if (live && ks == 0) {
            const Cx<R> cpl = cvt<R>(vn[i]);
#pragma unroll
            for (int gg = 0; gg < GC; ++gg) {
              const int g = gq * GC + gg;
              const Cx<R> y = acc[gg];
              const bool valid = g < gcount;
              const long long p = (long long)(g0 + g) * a.N + (long long)m * n + lo_c + i;
              if (fwd) {
                if (m < n - 1) {
                  Cx<R> f(0, 0);
                  if (valid) {
                    a.w[p] = y;
                    f = cvt<R>(reinterpret_cast<const c128*>(vin)[g * SM + i]);
                  }
                  xn[i * G + g] = f - cpl * y;
                } else {
                  if (valid) a.z[p] = cvt<double>(y);
                  xn[i * G + g] = cpl * y;
                }
              } else {
                Cx<R> u(0, 0);
                if (valid) {
                  u = reinterpret_cast<const Cx<R>*>(vin)[g * SM + i] - y;
                  a.z[p] = cvt<double>(u);
                }
                if (m > 0) xn[i * G + g] = cpl * u;
              }
            }
          }
        }
      }
      if (!alive && tid == 0) s_flags[0] = 1;
      __syncthreads();
    }
  }
  if (!GRID) cg::this_cluster().sync();   // no CTA leaves while others may still use the cluster
}

struct TmaConfig {
  bool ok, grid;
  int dC, C, G, nteams, KS;
  size_t smem;
};

static int ilog2i(int x) { int l = 0; while ((1 << (l + 1)) <= x) ++l; return l; }

// shared-memory plan for (dC, G, KS); returns total bytes
template <typename R>
static size_t plan(const hsweep_s* h, int dC, int G, int KS, TmaArgs<R>& a) {
  const size_t es = sizeof(Cx<R>);
  const int nl = 1 << (h->L - dC);
  const int slab_max = h->tree.maxsz(dC);
  const int rcap = std::max(1, h->rank_max);
  auto al = [](size_t x, size_t b) { return (x + b - 1) / b * b; };
  size_t o = 0;
  const size_t stage = al((size_t)h->slab_bytes_max[dC], 128);
  for (int b = 0; b < 2; ++b) { a.o_stage[b] = (unsigned)o; o += stage; }
  for (int b = 0; b < 2; ++b) { a.o_rowoff[b] = (unsigned)o; o += al((size_t)(h->L + 1) * slab_max * sizeof(int), 16); }
  for (int b = 0; b < 3; ++b) { a.o_trk[b] = (unsigned)o; o += al((size_t)(dC + 2 * nl) * sizeof(int), 16); }
  for (int b = 0; b < 3; ++b) { a.o_ro[b] = (unsigned)o; o += al((size_t)(nl + 1) * sizeof(long long), 16); }
  for (int b = 0; b < 2; ++b) { a.o_vin[b] = (unsigned)o; o += al((size_t)G * slab_max * sizeof(c128), 16); }
  for (int b = 0; b < 2; ++b) { a.o_vn[b] = (unsigned)o; o += al((size_t)slab_max * sizeof(c128), 16); }
  a.o_lo = (unsigned)o; o += al(h->nnodes * sizeof(int), 16);
  a.o_sz = (unsigned)o; o += al(h->nnodes * sizeof(int), 16);
  a.o_leafnode = (unsigned)o; o += al(slab_max * sizeof(int), 16);
  a.o_dtab = (unsigned)o; o += al(DT_SIZE * sizeof(int), 16);
  {
    long long wtot = 0;
    for (int d = 1; d <= h->L; ++d) {
      const int rows = d <= dC ? slab_max : h->tree.maxsz(d);
      const int nodes = d <= dC ? 1 : (1 << (d - dC));
      const int qcap = d <= dC ? rcap : std::min(rows, rcap);
      int kw = 1;
      const int kwmax = d <= dC ? 8 : 16;
      while (kw < qcap && kw < kwmax) kw <<= 1;
      wtot += (long long)nodes * ((qcap + kw - 1) / kw) * (G <= 5 ? 1 : G / 4);
    }
    a.o_wdesc = (unsigned)o; o += al((size_t)wtot * sizeof(int), 16);
  }
  a.o_boff = (unsigned)o; o += al((size_t)2 * nl * (h->L + 1) * sizeof(int), 16);
  for (int b = 0; b < 2; ++b) { a.o_x[b] = (unsigned)o; o += al((size_t)slab_max * G * es, 16); }
  a.o_qanc = (unsigned)o; o += al((size_t)std::max(1, dC) * rcap * G * es, 16);
  long long qloc = 0;
  for (int d = dC + 1; d <= h->L; ++d) qloc += (long long)(1 << (d - dC)) * std::min(h->tree.maxsz(d), rcap) * G;
  a.o_qloc = (unsigned)o; o += al((size_t)std::max(1LL, qloc) * es, 16);
  a.o_mbar = (unsigned)o; o += 16;
  a.o_flags = (unsigned)o; o += 16;
  a.stage_bytes = (unsigned)stage;
  a.nl = nl;
  a.slab_max = slab_max;
  a.rcap = rcap;
  a.KS = KS;
  return o;
}

template <typename R, int G, bool GRID>
static int max_clusters(const TmaConfig& cfg, int C, size_t smem);

template <typename R>
static int team_capacity(const hsweep_s* h, int C, int G, size_t smem) {
  if (C > 16) return 1;
  int k = 0;
  switch (G) {
    case 1: k = max_clusters<R, 1, false>(TmaConfig{}, C, smem); break;
    case 2: k = max_clusters<R, 2, false>(TmaConfig{}, C, smem); break;
    case 4: k = max_clusters<R, 4, false>(TmaConfig{}, C, smem); break;
    case 5: k = max_clusters<R, 5, false>(TmaConfig{}, C, smem); break;
    default: k = max_clusters<R, 8, false>(TmaConfig{}, C, smem); break;
  }
  if (k <= 0) k = std::max(1, h->num_sms / C);
  return k;
}

template <typename R>
static TmaConfig choose_tma(const hsweep_s* h, int nrhs) {
  TmaConfig best{};
  best.ok = false;
  double best_cost = 1e300;
  const size_t cap = 227 * 1024;
  const int C_pref = h->opt.team, G_pref = h->opt.groups;
  const bool fp64_small = h->prec == HSWEEP_FP64 && nrhs <= 2;
  const int cands_a[] = {16, 8, 4, 2, 1, 32, 64, 128};
  const int cands_b[] = {64, 32, 128, 16, 8, 4, 2, 1};
  const int* cands = fp64_small ? cands_b : cands_a;
  for (int ci = 0; ci < 8; ++ci) {
    const int C = cands[ci];
    if (C_pref > 0 && C != (1 << ilog2i(C_pref))) continue;
    if (C > h->nleaves || C > h->num_sms) continue;
    const int dC = ilog2i(C);
    const bool grid = C > 16;
    for (int G : {8, 5, 4, 2, 1}) {
      if (G_pref > 0 && G != G_pref) continue;
      for (int KS : {8}) {
        TmaArgs<R> a;
        const size_t smem = plan<R>(h, dC, G, KS, a);
        if (smem > cap) continue;
        const int teams_cap = grid ? 1 : team_capacity<R>(h, C, G, smem);
        const int ngroups = (nrhs + G - 1) / G;
        const int teams = std::min(ngroups, teams_cap);
        const int rounds = (ngroups + teams - 1) / teams;
        // rounds of 2n-1 dependent steps; a step costs a fixed latency plus work that
        // grows with the right-hand sides per team and shrinks with the CTAs per team
        const double step = 1.0 + 0.12 * G * (16.0 / C) * (grid ? 1.0 : 1.0) + (grid ? 1.5 : 0.0);
        const double cost = rounds * step;
        if (cost < best_cost - 1e-9) {
          best_cost = cost;
          best.ok = true;
          best.grid = grid;
          best.dC = dC;
          best.C = C;
          best.G = G;
          best.KS = KS;
          best.smem = smem;
          best.nteams = teams;
        }
        break;   // the largest KS that fits
      }
    }
    if (best.ok && C_pref == 0 && !fp64_small) break;   // prefer the first team size that fits
    if (best.ok && fp64_small) break;
  }
  return best;
}

template <typename R, int G, bool GRID>
static int launch_tma(hsweep_s* h, const TmaConfig& cfg, TmaArgs<R>& a) {
  auto kern = sweep_tma_kernel<R, G, GRID>;
  HSW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem));
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[1];
  lc.blockDim = dim3(kThreads);
  lc.dynamicSmemBytes = cfg.smem;
  lc.stream = h->stream;
  if (GRID) {
    lc.gridDim = dim3(cfg.C);
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
  } else {
    if (cfg.C > 8) HSW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    lc.gridDim = dim3(cfg.C * cfg.nteams);
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cfg.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
  }
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

template <typename R, int G, bool GRID>
static int max_clusters(const TmaConfig&, int C, size_t smem) {
  auto kern = sweep_tma_kernel<R, G, GRID>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[1];
  lc.blockDim = dim3(kThreads);
  lc.gridDim = dim3(C);
  lc.dynamicSmemBytes = smem;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  int k = 0;
  if (cudaOccupancyMaxActiveClusters(&k, kern, &lc) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return k;
}

template <typename R, bool GRID>
static int dispatch_tma(hsweep_s* h, const TmaConfig& cfg, TmaArgs<R>& a) {
  switch (cfg.G) {
    case 1: return launch_tma<R, 1, GRID>(h, cfg, a);
    case 2: return launch_tma<R, 2, GRID>(h, cfg, a);
    case 4: return launch_tma<R, 4, GRID>(h, cfg, a);
    case 5: return launch_tma<R, 5, GRID>(h, cfg, a);
    default: return launch_tma<R, 8, GRID>(h, cfg, a);
  }
}

static long long al256(long long x) { return (x + 255) / 256 * 256; }

// scratch of the TMA sweep: the w cache and the ancestors' exchange slots
template <typename R>
static void scratch_need(const hsweep_s* h, int nrhs, const TmaConfig& cfg, long long* w_bytes, long long* x_bytes) {
  const long long es = sizeof(Cx<R>);
  *w_bytes = (long long)nrhs * h->N * es;
  *x_bytes = 2LL * cfg.nteams * cfg.C * std::max(1, cfg.dC) * std::max(1, h->rank_max) * cfg.G * es;
}

template <typename R>
static int apply_tma_impl(hsweep_s* h, const c128* r, c128* z, int nrhs, bool* used, void* scratch,
                          size_t scratch_bytes) {
  *used = false;
  TmaConfig cfg = choose_tma<R>(h, nrhs);
  if (!cfg.ok) return HSWEEP_OK;
  const size_t es = sizeof(Cx<R>);
  long long wb, xb;
  scratch_need<R>(h, nrhs, cfg, &wb, &xb);
  void* wptr;
  void* xptr;
  if (scratch) {    // caller-provided scratch: nothing is allocated
    if ((size_t)(al256(wb) + al256(xb)) > scratch_bytes) return HSWEEP_ERR_ARG;
    wptr = scratch;
    xptr = (unsigned char*)scratch + al256(wb);
  } else {
    long long need_w = (long long)nrhs * h->N;
    if (need_w > h->wcache_cap) {
      hsw_release(h, h->d_wcache); h->d_wcache = nullptr; h->wcache_cap = 0;
      int rc = hsw_alloc(h, &h->d_wcache, (size_t)need_w * es);
      if (rc) return rc;
      h->wcache_cap = need_w;
    }
    long long need_x = xb / (long long)es;
    if (need_x > h->xch_cap) {
      hsw_release(h, h->d_xch); h->d_xch = nullptr; h->xch_cap = 0;
      int rc = hsw_alloc(h, &h->d_xch, (size_t)need_x * es);
      if (rc) return rc;
      h->xch_cap = need_x;
    }
    wptr = h->d_wcache;
    xptr = h->d_xch;
  }
  TmaArgs<R> a;
  plan<R>(h, cfg.dC, cfg.G, cfg.KS, a);
  a.n = h->n; a.L = h->L; a.leaf = h->leaf; a.nnodes = h->nnodes; a.dC = cfg.dC; a.C = cfg.C;
  a.nteams = cfg.nteams; a.nrhs = nrhs; a.ngroups = (nrhs + cfg.G - 1) / cfg.G;
  a.N = h->N; a.pack_stride = h->pack_stride;
  a.lo = h->d_lo; a.sz = h->d_sz; a.rank = h->d_rank; a.recoff = h->d_recoff;
  a.pack = reinterpret_cast<const Cx<R>*>(h->d_pack);
  a.north = h->d_north; a.r = r; a.z = z;
  a.w = reinterpret_cast<Cx<R>*>(wptr);
  a.xch = reinterpret_cast<Cx<R>*>(xptr);
  a.status = h->d_status; a.bar = h->d_bar;
  int rc;
  const bool prof = h->prof;
  if (scratch) h->prof = false;   // the no-allocation path creates no events
  if (cfg.grid) {
    if (cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), h->stream) != cudaSuccess) { h->prof = prof; return HSWEEP_ERR_CUDA; }
    rc = dispatch_tma<R, true>(h, cfg, a);
  } else {
    rc = dispatch_tma<R, false>(h, cfg, a);
  }
  h->prof = prof;
  if (rc == HSWEEP_OK) *used = true;
  return rc;
}

}  // namespace

int hsw_tma_plan(hsweep_s* h, int nrhs, long long* out) {
  TmaConfig cfg{};
  if (h->pack_valid && !h->slab_bytes_max.empty())
    cfg = h->prec == HSWEEP_FP64 ? choose_tma<double>(h, nrhs) : choose_tma<float>(h, nrhs);
  out[0] = cfg.ok ? 1 : 0; out[1] = cfg.C; out[2] = cfg.G; out[3] = cfg.nteams; out[4] = cfg.grid;
  out[5] = (long long)cfg.smem; out[6] = cfg.ok ? h->slab_bytes_max[cfg.dC] : 0; out[7] = cfg.KS;
  return HSWEEP_OK;
}

int hsw_apply_tma(hsweep_s* h, const c128* r, c128* z, int nrhs, bool* used, void* scratch, size_t scratch_bytes) {
  *used = false;
  if (!h->pack_valid || h->slab_bytes_max.empty()) return HSWEEP_OK;
  if (h->prec == HSWEEP_FP64) return apply_tma_impl<double>(h, r, z, nrhs, used, scratch, scratch_bytes);
  return apply_tma_impl<float>(h, r, z, nrhs, used, scratch, scratch_bytes);
}

// bytes of caller-provided scratch the TMA sweep needs for nrhs (0 if it would not be used)
size_t hsw_apply_tma_scratch_bytes(hsweep_s* h, int nrhs) {
  if (!h->pack_valid || h->slab_bytes_max.empty() || h->opt.sweep_kernel == 1) return 0;
  long long wb, xb;
  if (h->prec == HSWEEP_FP64) {
    TmaConfig cfg = choose_tma<double>(h, nrhs);
    if (!cfg.ok) return 0;
    scratch_need<double>(h, nrhs, cfg, &wb, &xb);
  } else {
    TmaConfig cfg = choose_tma<float>(h, nrhs);
    if (!cfg.ok) return 0;
    scratch_need<float>(h, nrhs, cfg, &wb, &xb);
  }
  return (size_t)(al256(wb) + al256(xb));
}
