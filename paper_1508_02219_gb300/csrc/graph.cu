// Graph-based compression of VBARMS on the GPU (Section 2.2, Alg. 1) with a
// minimum block density mu.
//
//   G1  closed neighbourhoods adj(i) of the graph of A + A^T: the pairs
//       (i, i), (i, j), (j, i) of every stored a_ij, radix-sorted and made
//       unique, give a symmetric CSR with sorted rows
//   G2  the checksum scan: a vertex's class is the set of vertices with an
//       identical adj; vertices are sorted by a hash of adj (any exact hash
//       gives the same classes as the printed checksum, since classes are
//       decided by comparing the lists), and within a run of equal hashes
//       each vertex finds the first vertex with the same list; a class is
//       numbered by its smallest vertex
//   G3  the merge pass: supernodes in ascending order of their smallest
//   G4  vertex take their turn; the candidates of X are the supernodes owning
//       a vertex of adj(X) when the turn starts, in ascending order of their
//       smallest vertex; Z merges into X when the density N/T of the merged
//       supernode's block row and column reaches mu, with
//       T = 2 |adj(S)| |S| - |S|^2 and N = 2 sum_v |adj(v)| - sum_v |adj(v) n S|
//       (S = X u Z).  Every turn reads what the earlier ones changed (owners,
//       adjacencies, densities), so this pass is one warp walking the turns
//       in order, each turn's set operations spread over its lanes.
//   G5  blocks in ascending order of their smallest vertex, vertices
//       ascending; the VBCSR assembly of the angle-based compression.
#include <algorithm>
#include <climits>

#include "internal.h"

namespace vb {
namespace {

// ---- G1 -------------------------------------------------------------------
__global__ void k_pairs(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                        unsigned long long* __restrict__ key) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  const int64_t nnz = rowptr[n];
  for (int64_t i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += (int64_t)gridDim.x * wpb) {
    if (lane == 0) key[i] = (unsigned long long)i * (unsigned long long)n + (unsigned long long)i;
    for (int64_t q = rowptr[i] + lane; q < rowptr[i + 1]; q += 32) {
      const unsigned long long j = (unsigned long long)colind[q];
      key[n + q] = (unsigned long long)i * (unsigned long long)n + j;
      key[n + nnz + q] = j * (unsigned long long)n + (unsigned long long)i;
    }
  }
}

// first[k] = 1 when key[k] starts a run of equal keys.
__global__ void k_first(int64_t m, const unsigned long long* __restrict__ key, int32_t* __restrict__ first) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    first[k] = (k == 0 || key[k] != key[k - 1]) ? 1 : 0;
}

// The unique pairs: adjcol, and the row counts.
__global__ void k_unique(int64_t m, int64_t n, const unsigned long long* __restrict__ key,
                         const int32_t* __restrict__ first, const int64_t* __restrict__ pos,
                         int32_t* __restrict__ adjcol, int32_t* __restrict__ rowcnt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    if (first[k]) {
      const unsigned long long x = key[k];
      const int64_t i = (int64_t)(x / (unsigned long long)n);
      adjcol[pos[k]] = (int32_t)(x - (unsigned long long)i * (unsigned long long)n);
      atomicAdd(&rowcnt[i], 1);
    }
}

// ---- G2 -------------------------------------------------------------------
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

// key[v] = (32-bit hash of list v) << 32 | v, warp per list (the lists of a
// CSR: closed neighbourhoods here, row patterns for the two-pass variant).
__global__ void k_adj_hash(int64_t n, const int64_t* __restrict__ adjptr, const int32_t* __restrict__ adjcol,
                           unsigned long long* __restrict__ key) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t v = blockIdx.x * wpb + (threadIdx.x >> 5); v < n; v += (int64_t)gridDim.x * wpb) {
    unsigned long long h = 0;
    for (int64_t q = adjptr[v] + lane; q < adjptr[v + 1]; q += 32)
      h += mix64((unsigned long long)(unsigned)adjcol[q] * 0x9e3779b97f4a7c15ull + (unsigned long long)(q - adjptr[v]));
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    h = mix64(h ^ (unsigned long long)(adjptr[v + 1] - adjptr[v]));
    if (lane == 0) key[v] = ((h >> 32) << 32) | (unsigned long long)v;
  }
}

__device__ bool same_adj(const int64_t* __restrict__ adjptr, const int32_t* __restrict__ adjcol, int64_t u,
                         int64_t v) {
  const int64_t a = adjptr[u], la = adjptr[u + 1] - a, b = adjptr[v], lb = adjptr[v + 1] - b;
  if (la != lb) return false;
  for (int64_t q = 0; q < la; ++q)
    if (adjcol[a + q] != adjcol[b + q]) return false;
  return true;
}

// Sorted keys (hash, vertex): leader[v] = the first vertex of v's hash run
// whose list equals v's (the smallest vertex of v's class of identical lists).
__global__ void k_class_leader(int64_t n, const unsigned long long* __restrict__ skey,
                               const int64_t* __restrict__ adjptr, const int32_t* __restrict__ adjcol,
                               int32_t* __restrict__ leader) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long h = skey[k] >> 32;
    const int64_t v = (int64_t)(skey[k] & 0xffffffffull);
    int64_t r = k;
    while (r > 0 && (skey[r - 1] >> 32) == h) --r;
    int64_t lead = v;
    for (int64_t q = r; q < k; ++q) {
      const int64_t u = (int64_t)(skey[q] & 0xffffffffull);
      if (same_adj(adjptr, adjcol, u, v)) {
        lead = u;
        break;
      }
    }
    leader[v] = (int32_t)lead;
  }
}

__global__ void k_is_self(int64_t n, const int32_t* __restrict__ leader, int32_t* __restrict__ flag) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    flag[v] = leader[v] == (int32_t)v ? 1 : 0;
}

// Supernode of every vertex, and the initial supernode data: size, the sum of
// |adj(v)|, the smallest vertex, the adjacency (that of the smallest vertex).
__global__ void k_super_init(int64_t n, const int32_t* __restrict__ leader, const int64_t* __restrict__ lscan,
                             const int64_t* __restrict__ adjptr, int32_t* __restrict__ owner,
                             int32_t* __restrict__ msize, long long* __restrict__ deg, int32_t* __restrict__ minv,
                             int64_t* __restrict__ aoff, int32_t* __restrict__ alen) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t z = (int32_t)lscan[leader[v]];
    owner[v] = z;
    atomicAdd(&msize[z], 1);
    atomicAdd((unsigned long long*)&deg[z], (unsigned long long)(adjptr[v + 1] - adjptr[v]));
    if (leader[v] == (int32_t)v) {
      minv[z] = (int32_t)v;
      aoff[z] = adjptr[v];
      alen[z] = (int32_t)(adjptr[v + 1] - adjptr[v]);
    }
  }
}

// inner[z] = sum over v in z of |adj(v) n z| (warp per vertex).
__global__ void k_super_inner(int64_t n, const int64_t* __restrict__ adjptr, const int32_t* __restrict__ adjcol,
                              const int32_t* __restrict__ owner, long long* __restrict__ inner) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t v = blockIdx.x * wpb + (threadIdx.x >> 5); v < n; v += (int64_t)gridDim.x * wpb) {
    const int32_t z = owner[v];
    int c = 0;
    for (int64_t q = adjptr[v] + lane; q < adjptr[v + 1]; q += 32) c += owner[adjcol[q]] == z ? 1 : 0;
    c = warp_sum_i(c);
    if (lane == 0 && c) atomicAdd((unsigned long long*)&inner[z], (unsigned long long)c);
  }
}

// Member lists, linked in ascending vertex order: vertices sorted by
// (owner, vertex) in order[].
__global__ void k_link_members(int64_t n, const int32_t* __restrict__ order, const int32_t* __restrict__ owner,
                               int32_t* __restrict__ mhead, int32_t* __restrict__ mtail, int32_t* __restrict__ mnext) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = order[k], z = owner[v];
    const bool head = k == 0 || owner[order[k - 1]] != z;
    const bool tail = k == n - 1 || owner[order[k + 1]] != z;
    if (head) mhead[z] = v;
    if (tail) mtail[z] = v;
    mnext[v] = tail ? -1 : order[k + 1];
  }
}

// ---- G3/G4: the merge pass, one warp ---------------------------------------
struct MergeState {
  int64_t nsup;
  const int64_t* adjptr;  // static closed neighbourhoods
  const int32_t* adjcol;
  int32_t* owner;         // [n]
  int32_t* minv;          // [nsup] smallest vertex
  int32_t* msize;         // [nsup]
  long long* deg;         // [nsup] sum of |adj(v)|
  long long* inner;       // [nsup] sum of |adj(v) n X|
  int32_t* alive;         // [nsup]
  int64_t* aoff;          // [nsup] adjacency of the supernode in apool
  int32_t* alen;          // [nsup]
  int32_t* apool;         // static adjcol, then room for grown adjacencies
  int64_t apool_cap;
  unsigned long long* apool_top;
  int32_t* mhead;         // [nsup] member lists
  int32_t* mtail;
  int32_t* mnext;         // [n]
  int32_t* vmark;         // [n] turn stamp of the vertices in adj(X)
  int32_t* smark;         // [nsup] turn stamp of the candidates
  int32_t* cand;          // [ccap] candidates of the current turn
  int64_t ccap;
  double mu;
};

__global__ void __launch_bounds__(32, 1) k_graph_merge(MergeState S, int* st) {
  const int lane = threadIdx.x;
  __shared__ unsigned long long sortbuf[1024];
  for (int64_t x = 0; x < S.nsup; ++x) {
    if (!S.alive[x]) continue;
    const int32_t stamp = (int32_t)(x + 1);
    // the vertices of adj(X) are stamped; the candidates are their owners
    // other than X, each taken once
    int ncand = 0;
    {
      const int64_t a0 = S.aoff[x];
      const int len = S.alen[x];
      for (int base = 0; base < len; base += 32) {
        const int q = base + lane;
        bool isc = false;
        int32_t z = -1;
        if (q < len) {
          const int32_t u = S.apool[a0 + q];
          S.vmark[u] = stamp;
          z = S.owner[u];
          if (z != (int32_t)x && atomicExch(&S.smark[z], stamp) != stamp) isc = true;
        }
        const unsigned b = __ballot_sync(0xffffffffu, isc);
        if (isc) {
          const int pos = ncand + __popc(b & ((1u << lane) - 1u));
          if (pos < S.ccap) S.cand[pos] = z;
        }
        ncand += __popc(b);
      }
      __syncwarp();
    }
    if (ncand > S.ccap) {
      if (lane == 0) dev_fail(st, DEV_OVERFLOW);
      return;
    }
    // candidates in ascending order of their smallest vertex
    if (ncand > 1) {
      unsigned long long* buf = sortbuf;
      int n2 = 1;
      while (n2 < ncand) n2 <<= 1;
      if (n2 > 1024) {
        if (lane == 0) dev_fail(st, DEV_OVERFLOW);
        return;
      }
      for (int p = lane; p < n2; p += 32)
        buf[p] = p < ncand ? ((unsigned long long)(unsigned)S.minv[S.cand[p]] << 32) | (unsigned)S.cand[p] : ~0ull;
      __syncwarp();
      for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int e = lane; e < n2; e += 32) {
            const int f = e ^ j;
            if (f > e) {
              const unsigned long long u = buf[e], v = buf[f];
              if ((u > v) == ((e & k) == 0)) {
                buf[e] = v;
                buf[f] = u;
              }
            }
          }
          __syncwarp();
        }
      for (int p = lane; p < ncand; p += 32) S.cand[p] = (int32_t)(buf[p] & 0xffffffffu);
      __syncwarp();
    }
    for (int c = 0; c < ncand; ++c) {
      const int32_t z = S.cand[c];
      // |adj(X) u adj(Z)|: the vertices of adj(Z) not stamped by X
      const int64_t z0 = S.aoff[z];
      const int zlen = S.alen[z];
      int fresh = 0;
      for (int q = lane; q < zlen; q += 32) fresh += S.vmark[S.apool[z0 + q]] != stamp ? 1 : 0;
      fresh = warp_sum_i(fresh);
      // cross = sum over v in Z of |adj(v) n X|
      long long cross = 0;
      for (int32_t v = S.mhead[z]; v >= 0; v = S.mnext[v]) {
        int cv = 0;
        for (int64_t q = S.adjptr[v] + lane; q < S.adjptr[v + 1]; q += 32) cv += S.owner[S.adjcol[q]] == (int32_t)x;
        cross += warp_sum_i(cv);
      }
      const long long sz = (long long)S.msize[x] + S.msize[z];
      const long long un = (long long)S.alen[x] + fresh;
      const long long T = 2 * un * sz - sz * sz;
      const long long N = 2 * (S.deg[x] + S.deg[z]) - (S.inner[x] + S.inner[z] + 2 * cross);
      if (!((double)N >= S.mu * (double)T)) continue;
      // merge Z into X: owners, members, adjacency (X's list grows by the
      // unstamped vertices of adj(Z), copied to fresh pool space), counts
      for (int32_t v = S.mhead[z]; v >= 0; v = S.mnext[v])
        if (lane == 0) S.owner[v] = (int32_t)x;
      unsigned long long top = 0;
      const int nlen = S.alen[x] + fresh;
      if (lane == 0) top = atomicAdd(S.apool_top, (unsigned long long)nlen);
      top = __shfl_sync(0xffffffffu, top, 0);
      if ((int64_t)top + nlen > S.apool_cap) {
        if (lane == 0) dev_fail(st, DEV_OVERFLOW);
        return;
      }
      const int64_t x0 = S.aoff[x];
      const int xlen = S.alen[x];
      for (int q = lane; q < xlen; q += 32) S.apool[top + q] = S.apool[x0 + q];
      int w = xlen;
      for (int base = 0; base < zlen; base += 32) {
        const int q = base + lane;
        int32_t u = -1;
        bool add = false;
        if (q < zlen) {
          u = S.apool[z0 + q];
          add = S.vmark[u] != stamp;
        }
        const unsigned b = __ballot_sync(0xffffffffu, add);
        if (add) S.apool[top + w + __popc(b & ((1u << lane) - 1u))] = u;
        w += __popc(b);
        __syncwarp();
        if (add) S.vmark[u] = stamp;
      }
      __syncwarp();
      if (lane == 0) {
        S.aoff[x] = (int64_t)top;
        S.alen[x] = nlen;
        S.mnext[S.mtail[x]] = S.mhead[z];
        S.mtail[x] = S.mtail[z];
        S.msize[x] += S.msize[z];
        S.deg[x] += S.deg[z];
        S.inner[x] += S.inner[z] + 2 * cross;
        S.minv[x] = min(S.minv[x], S.minv[z]);
        S.alive[z] = 0;
      }
      __syncwarp();
    }
  }
}

// Final grouping: the smallest vertex of every vertex's supernode.
__global__ void k_final_leader(int64_t n, const int32_t* __restrict__ owner, const int32_t* __restrict__ minv,
                               int32_t* __restrict__ lead) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    lead[v] = minv[owner[v]];
}

__global__ void k_block_index(int64_t n, const int32_t* __restrict__ lead, const int64_t* __restrict__ lscan,
                              int32_t* __restrict__ blk, int32_t* __restrict__ bsz,
                              unsigned long long* __restrict__ key) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = (int32_t)lscan[lead[v]];
    blk[v] = b;
    atomicAdd(&bsz[b], 1);
    key[v] = ((unsigned long long)(unsigned)b << 32) | (unsigned long long)v;
  }
}

// perm (vertices by block, ascending) and each vertex's place in its block.
__global__ void k_perm_offin(int64_t n, const unsigned long long* __restrict__ skey, const int64_t* __restrict__ boff,
                             const int32_t* __restrict__ blk, int32_t* __restrict__ perm,
                             int32_t* __restrict__ offin) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = (int32_t)(skey[k] & 0xffffffffull);
    perm[k] = v;
    offin[v] = (int32_t)(k - boff[blk[v]]);
  }
}

__global__ void k_fill_i32(int64_t n, int32_t v, int32_t* __restrict__ a) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    a[k] = v;
}

__global__ void k_owner_key(int64_t n, const int32_t* __restrict__ owner, unsigned long long* __restrict__ key) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    key[v] = ((unsigned long long)(unsigned)owner[v] << 32) | (unsigned long long)v;
}

__global__ void k_key_low(int64_t n, const unsigned long long* __restrict__ key, int32_t* __restrict__ out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    out[v] = (int32_t)(key[v] & 0xffffffffull);
}

int bits_for(unsigned long long x) {
  int b = 0;
  while (b < 64 && (x >> b) != 0) ++b;
  return std::max(b, 1);
}

}  // namespace

void list_classes(int64_t n, const int64_t* ptr, const int32_t* col, int32_t* leader, cudaStream_t s) {
  if (n == 0) return;
  DBuf<unsigned long long> hk(n, s);
  launch(k_adj_hash, grid_for(n, 8), 256, 0, s, n, ptr, col, hk.p);
  VB_LAUNCH_CHECK();
  radix_sort_u64(hk, nullptr, n, 64, s);
  launch(k_class_leader, grid_for(n, 256), 256, 0, s, n, hk.p, ptr, col, leader);
  VB_LAUNCH_CHECK();
}

void graph_compress_device(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val, double mu,
                           cudaStream_t s, int* dst, Compressed& out) {
  out.n = n;
  out.nnz = n ? d2h(rowptr + n, s) : 0;
  const int64_t nnz = out.nnz;
  {
    DBuf<int32_t> len(std::max<int64_t>(n, 1), s);
    if (n) validate_csr(n, rowptr, colind, len.p, s, dst);
  }
  check_status(dst, s, "vbarms_compress_graph: CSR validation");
  if (n == 0) {
    assemble_from_leaders(0, rowptr, colind, val, nullptr, s, dst, out);
    return;
  }
  // G1: symmetric closed adjacency, rows sorted
  const int64_t m = n + 2 * nnz;
  const int kbits = bits_for((unsigned long long)n * (unsigned long long)n);
  DBuf<unsigned long long> pk(m, s);
  launch(k_pairs, grid_for(n, 8), 256, 0, s, n, rowptr, colind, pk.p);
  VB_LAUNCH_CHECK();
  radix_sort_u64(pk, nullptr, m, kbits, s);
  DBuf<int32_t> first(m, s), rowcnt(n, s);
  DBuf<int64_t> pos(m + 1, s), adjptr(n + 1, s);
  launch(k_first, grid_for(m, 256), 256, 0, s, m, pk.p, first.p);
  VB_LAUNCH_CHECK();
  scan_i32_to_i64(first.p, pos.p, m, s);
  const int64_t E = d2h(pos.p + m, s);
  rowcnt.zero();
  // the adjacency pool: the static lists, then room for the merge pass
  const int64_t apool_cap = E + std::max<int64_t>(4 * E, 1 << 20);
  DBuf<int32_t> apool(apool_cap, s);
  launch(k_unique, grid_for(m, 256), 256, 0, s, m, n, pk.p, first.p, pos.p, apool.p, rowcnt.p);
  VB_LAUNCH_CHECK();
  scan_i32_to_i64(rowcnt.p, adjptr.p, n, s);
  pk.release();
  first.release();
  pos.release();
  rowcnt.release();
  // G2: classes of identical adjacency
  DBuf<int32_t> leader(n, s), isl(n, s);
  list_classes(n, adjptr.p, apool.p, leader.p, s);
  launch(k_is_self, grid_for(n, 256), 256, 0, s, n, leader.p, isl.p);
  VB_LAUNCH_CHECK();
  DBuf<int64_t> lscan(n + 1, s);
  scan_i32_to_i64(isl.p, lscan.p, n, s);
  const int64_t nsup = d2h(lscan.p + n, s);
  DBuf<int32_t> owner(n, s), msize(nsup, s), minv(nsup, s), alen(nsup, s), alive(nsup, s), mhead(nsup, s),
      mtail(nsup, s), mnext(n, s), vmark(n, s), smark(nsup, s);
  DBuf<long long> deg(nsup, s), inner(nsup, s);
  DBuf<int64_t> aoff(nsup, s);
  msize.zero();
  deg.zero();
  inner.zero();
  vmark.zero();
  smark.zero();
  {
    if (nsup) {
      launch(k_fill_i32, grid_for(nsup, 256), 256, 0, s, nsup, 1, alive.p);
      VB_LAUNCH_CHECK();
    }
    launch(k_super_init, grid_for(n, 256), 256, 0, s, n, leader.p, lscan.p, adjptr.p, owner.p, msize.p, deg.p,
           minv.p, aoff.p, alen.p);
    VB_LAUNCH_CHECK();
    launch(k_super_inner, grid_for(n, 8), 256, 0, s, n, adjptr.p, apool.p, owner.p, inner.p);
    VB_LAUNCH_CHECK();
    DBuf<unsigned long long> ok(n, s);
    launch(k_owner_key, grid_for(n, 256), 256, 0, s, n, owner.p, ok.p);
    VB_LAUNCH_CHECK();
    radix_sort_u64(ok, nullptr, n, 32 + bits_for((unsigned long long)nsup), s);
    DBuf<int32_t> order(n, s);
    launch(k_key_low, grid_for(n, 256), 256, 0, s, n, ok.p, order.p);
    VB_LAUNCH_CHECK();
    launch(k_link_members, grid_for(n, 256), 256, 0, s, n, order.p, owner.p, mhead.p, mtail.p, mnext.p);
    VB_LAUNCH_CHECK();
    VB_CUDA(cudaStreamSynchronize(s));
  }
  leader.release();
  isl.release();
  // G3/G4: the merge pass
  const int64_t ccap = std::min<int64_t>(std::max<int64_t>(nsup, 1), 1024);
  DBuf<int32_t> cand(ccap, s);
  DBuf<unsigned long long> top(1, s);
  h2d(top.p, reinterpret_cast<const unsigned long long*>(&E), 1, s);
  MergeState S{nsup,    adjptr.p, apool.p, owner.p, minv.p, msize.p,  deg.p,  inner.p,
               alive.p, aoff.p,   alen.p,  apool.p, apool_cap, top.p, mhead.p, mtail.p,
               mnext.p, vmark.p,  smark.p, cand.p,  ccap,    mu};
  if (nsup) {
    launch(k_graph_merge, 1, 32, 0, s, S, dst);
    VB_LAUNCH_CHECK();
  }
  if (d2h(dst, s) == DEV_OVERFLOW) {
    VB_CUDA(cudaMemsetAsync(dst, 0, sizeof(int), s));
    fail(VB_ENOMEM, "vbarms_compress_graph: a supernode's candidates or the adjacency pool exceed their capacity");
  }
  check_status(dst, s, "vbarms_compress_graph: merge pass");
  // G5: blocks by smallest vertex, vertices ascending
  DBuf<int32_t> lead(n, s);
  launch(k_final_leader, grid_for(n, 256), 256, 0, s, n, owner.p, minv.p, lead.p);
  VB_LAUNCH_CHECK();
  assemble_from_leaders(n, rowptr, colind, val, lead.p, s, dst, out);
}

void assemble_from_leaders(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
                           const int32_t* lead, cudaStream_t s, int* dst, Compressed& out) {
  if (n == 0) {
    DBuf<int32_t> bsz;
    DBuf<int64_t> boff(1, s);
    boff.zero();
    out.perm.alloc(0, s);
    assemble_vbcsr(0, rowptr, colind, val, 0, bsz, boff, nullptr, nullptr, s, dst, out);
    return;
  }
  DBuf<int32_t> isl2(n, s), blk(n, s), offin(n, s);
  launch(k_is_self, grid_for(n, 256), 256, 0, s, n, lead, isl2.p);
  VB_LAUNCH_CHECK();
  DBuf<int64_t> ls2(n + 1, s);
  scan_i32_to_i64(isl2.p, ls2.p, n, s);
  const int64_t p = d2h(ls2.p + n, s);
  DBuf<int32_t> bsz(p, s);
  bsz.zero();
  DBuf<unsigned long long> bk(n, s);
  launch(k_block_index, grid_for(n, 256), 256, 0, s, n, lead, ls2.p, blk.p, bsz.p, bk.p);
  VB_LAUNCH_CHECK();
  radix_sort_u64(bk, nullptr, n, 32 + bits_for((unsigned long long)p), s);
  DBuf<int64_t> boff(p + 1, s);
  scan_i32_to_i64(bsz.p, boff.p, p, s);
  out.perm.alloc(n, s);
  launch(k_perm_offin, grid_for(n, 256), 256, 0, s, n, bk.p, boff.p, blk.p, out.perm.p, offin.p);
  VB_LAUNCH_CHECK();
  assemble_vbcsr(n, rowptr, colind, val, p, bsz, boff, blk.p, offin.p, s, dst, out);
}

}  // namespace vb
