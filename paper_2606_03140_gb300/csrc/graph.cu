// Atom graph, recursive coordinate bisection and one-hop halos on the GPU.
//
// Graph (Sec. "Determining the Subgraphs", Fig. 1a/e; Sec. "Dynamic Graph Adaption"):
// edge (I, J), I != J, when the minimum-image distance is below r_G or when the
// atom-condensed density graph of the previous step exceeds tau in either direction.
// The distance test uses separately rounded IEEE operations (no contraction into fused
// multiply-adds) so the integer result is reproducible bit for bit:
//   dx = (x_J - x_I) - L * rint((x_J - x_I) / L),  r2 = (dx*dx + dy*dy) + dz*dz < r_G*r_G.
// Neighbour search uses a cell list with cells wider than r_G (one warp per atom over the
// flattened candidates of the 27 neighbour cells); every row is sorted and de-duplicated in
// shared memory, then compacted into CSR.
//
// Cores (Fig. 1b): recursive coordinate bisection of the wrapped coordinates
// w = x - L * floor(x / L).  The split sizes follow from integers only
// (floor(c * floor(p/2) / p) atoms take floor(p/2) cores), so the host knows the tree;
// each level sorts every segment by (w_axis, atom index) along its widest axis (first
// axis on ties) in one CTA.  Halo (Fig. 1c): graph neighbours of core atoms outside the
// core, ascending, from a per-core bitmap.
#include "graph.cuh"

#include <cmath>

namespace sedacs {

namespace {

__device__ __forceinline__ double wrap1(double x, double L) {
  return __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
}

__device__ __forceinline__ double min_image_r2(const double* R, int i, int j, const double* box) {
  double r2 = 0.0;
  double d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double dx = __dsub_rn(R[3 * j + a], R[3 * i + a]);
    d[a] = __dsub_rn(dx, __dmul_rn(box[a], rint(__ddiv_rn(dx, box[a]))));
  }
  r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
  return r2;
}

struct CellGrid {
  int nc[3];
  double cw[3];
  double box[3];
  int brute;   // 1: fewer than 3 cells on an axis, test every atom
  int exact;   // 1: separately rounded FP64 test (bit-reproducible); 0: FP32 test (pair lists)
};

__device__ __forceinline__ float min_image_r2_f(const double* R, int i, int j, const double* box) {
  float d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float dx = (float)(R[3 * j + a] - R[3 * i + a]);
    const float L = (float)box[a];
    dx -= L * rintf(dx / L);
    d[a] = dx;
  }
  return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

__global__ void cell_assign_kernel(const double* R, int N, CellGrid g, int* cell_of, int* cell_count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double w = wrap1(R[3 * i + a], g.box[a]);
    int k = (int)floor(w / g.cw[a]);
    c[a] = min(max(k, 0), g.nc[a] - 1);
  }
  const int cid = (c[0] * g.nc[1] + c[1]) * g.nc[2] + c[2];
  cell_of[i] = cid;
  atomicAdd(&cell_count[cid], 1);
}

__global__ void cell_fill_kernel(const int* cell_of, int N, const int* cell_start, int* cell_fill, int* cell_atoms) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int c = cell_of[i];
  const int slot = atomicAdd(&cell_fill[c], 1);
  cell_atoms[cell_start[c] + slot] = i;
}

// Warp per atom i: the candidates (atoms of the 27 cells around i's cell, or every atom when
// the grid is too coarse) are flattened, lane l takes candidates l, l + 32, ...; the cell of a
// flat index comes from a shuffle scan of the 27 cell counts and a shuffle binary search.
// f(j, hit) is called by all lanes together once per round (hit false on idle lanes).
template <typename F>
__device__ __forceinline__ void warp_distance_scan(const double* R, int N, int i, const CellGrid& g,
                                                   const int* cell_of, const int* cell_start, const int* cell_count,
                                                   const int* cell_atoms, double rg2, int lane, F f) {
  const double box[3] = {g.box[0], g.box[1], g.box[2]};
  const float rg2f = (float)rg2;
  auto within = [&](int j) {
    return g.exact ? (min_image_r2(R, i, j, box) < rg2) : (min_image_r2_f(R, i, j, box) < rg2f);
  };
  if (g.brute) {
    for (int b = 0; b < N; b += 32) {
      const int j = b + lane;
      f(j, j < N && j != i && within(j));
    }
    return;
  }
  const int cid = cell_of[i];
  const int cz = cid % g.nc[2], cy = (cid / g.nc[2]) % g.nc[1], cx = cid / (g.nc[2] * g.nc[1]);
  int st = 0, cnt = 0;
  if (lane < 27) {
    const int x = (cx + lane / 9 - 1 + g.nc[0]) % g.nc[0];
    const int y = (cy + (lane / 3) % 3 - 1 + g.nc[1]) % g.nc[1];
    const int z = (cz + lane % 3 - 1 + g.nc[2]) % g.nc[2];
    const int c = (x * g.nc[1] + y) * g.nc[2] + z;
    st = cell_start[c];
    cnt = cell_count[c];
  }
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int excl = incl - cnt;
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  for (int b = 0; b < total; b += 32) {
    const int t = b + lane;
    int lo = 0;                                   // largest cell q < 27 with excl[q] <= t
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int c = lo + step;
      const int ex = __shfl_sync(0xffffffffu, excl, c & 31);
      if (c < 27 && ex <= t) lo = c;
    }
    const int s0 = __shfl_sync(0xffffffffu, st, lo);
    const int e0 = __shfl_sync(0xffffffffu, excl, lo);
    int j = -1;
    if (t < total) j = cell_atoms[s0 + (t - e0)];
    f(j, t < total && j != i && within(j));
  }
}

__global__ void count_dist_kernel(const double* R, int N, CellGrid g, const int* cell_of, const int* cell_start,
                                  const int* cell_count, const int* cell_atoms, double rg2, int* cnt) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= N) return;
  int n = 0;
  warp_distance_scan(R, N, i, g, cell_of, cell_start, cell_count, cell_atoms, rg2, lane,
                     [&](int, bool hit) { n += __popc(__ballot_sync(0xffffffffu, hit)); });
  if (lane == 0) cnt[i] = n;
}

__global__ void count_gd_kernel(const long long* gptr, const int* gcol, const double* gval, int N, double tau,
                                int* cnt) {
  const int i = blockIdx.x;
  for (long long p = gptr[i] + threadIdx.x; p < gptr[i + 1]; p += blockDim.x) {
    const int j = gcol[p];
    if (j != i && j >= 0 && j < N && gval[p] > tau) {
      atomicAdd(&cnt[i], 1);
      atomicAdd(&cnt[j], 1);
    }
  }
}

__global__ void fill_dist_kernel(const double* R, int N, CellGrid g, const int* cell_of, const int* cell_start,
                                 const int* cell_count, const int* cell_atoms, double rg2, const long long* cptr,
                                 int* fillc, int* cand) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= N) return;
  const long long base = cptr[i];
  int n = 0;
  warp_distance_scan(R, N, i, g, cell_of, cell_start, cell_count, cell_atoms, rg2, lane, [&](int j, bool hit) {
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (hit) cand[base + n + __popc(m & ((1u << lane) - 1u))] = j;
    n += __popc(m);
  });
  if (lane == 0) fillc[i] = n;
}

// exclusive scan of the cell counts (one block)
__global__ void cell_scan_kernel(const int* count, int ncell, int* start) {
  __shared__ int part[1024];
  const int per = (ncell + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per, b1 = min(ncell, b0 + per);
  int s = 0;
  for (int c = b0; c < b1; ++c) s += count[c];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const int v = part[t];
      part[t] = acc;
      acc += v;
    }
    start[ncell] = acc;
  }
  __syncthreads();
  int acc = part[threadIdx.x];
  for (int c = b0; c < b1; ++c) {
    start[c] = acc;
    acc += count[c];
  }
}

// Candidates from a previous (symmetric) graph: every edge is kept (used while the SCC grows
// its graph, edges added and not removed).
__global__ void count_prev_kernel(const long long* pptr, int N, int* cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) cnt[i] += (int)(pptr[i + 1] - pptr[i]);
}

__global__ void fill_prev_kernel(const long long* pptr, const int* pcol, int N, const long long* cptr, int* fillc,
                                 int* cand) {
  const int i = blockIdx.x;
  const long long b = pptr[i], e = pptr[i + 1];
  const int base = fillc[i];
  for (long long p = b + threadIdx.x; p < e; p += blockDim.x) cand[cptr[i] + base + (p - b)] = pcol[p];
  __syncthreads();
  if (threadIdx.x == 0) fillc[i] = base + (int)(e - b);
}

__global__ void fill_gd_kernel(const long long* gptr, const int* gcol, const double* gval, int N, double tau,
                               const long long* cptr, int* fillc, int* cand) {
  const int i = blockIdx.x;
  for (long long p = gptr[i] + threadIdx.x; p < gptr[i + 1]; p += blockDim.x) {
    const int j = gcol[p];
    if (j != i && j >= 0 && j < N && gval[p] > tau) {
      cand[cptr[i] + atomicAdd(&fillc[i], 1)] = j;
      cand[cptr[j] + atomicAdd(&fillc[j], 1)] = i;
    }
  }
}

// Sort one row's candidates, drop duplicates, write the unique count (sorted in place).
__global__ void row_unique_kernel(const long long* cptr, int* cand, int* ucnt, int* err, int cap) {
  extern __shared__ int sk[];
  const int i = blockIdx.x;
  const long long base = cptr[i];
  const int n = (int)(cptr[i + 1] - base);
  if (n > cap) {
    if (threadIdx.x == 0) { atomicOr(err, kErrCapacity); ucnt[i] = 0; }
    return;
  }
  int P2 = 1;
  while (P2 < n) P2 <<= 1;
  for (int t = threadIdx.x; t < P2; t += blockDim.x) sk[t] = (t < n) ? cand[base + t] : 0x7fffffff;
  __syncthreads();
  for (int k = 2; k <= P2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < P2; t += blockDim.x) {
        const int u = t ^ j;
        if (u > t) {
          const bool up = (t & k) == 0;
          const int a = sk[t], b = sk[u];
          if ((a > b) == up) { sk[t] = b; sk[u] = a; }
        }
      }
      __syncthreads();
    }
  if (threadIdx.x == 0) {
    int m = 0;
    for (int t = 0; t < n; ++t)
      if (t == 0 || sk[t] != sk[t - 1]) cand[base + m++] = sk[t];
    ucnt[i] = m;
  }
}

__global__ void compact_kernel(const long long* cptr, const int* cand, const long long* row_ptr, int N, int* col) {
  const int i = blockIdx.x;
  const long long s = cptr[i], d = row_ptr[i];
  const int n = (int)(row_ptr[i + 1] - d);
  for (int t = threadIdx.x; t < n; t += blockDim.x) col[d + t] = cand[s + t];
}

// Weighted two-hop rule (Sec. "Dynamic Graph Adaption", Eq. "Graph_Adaptation"), one block per
// atom I: P_IJ = sum over K in {I} and I's neighbour row (ascending K) of G^N_IK G^D_KJ, with
// G^N_II = 1 and G^N_IK = exp(-alpha R_IK^2), accumulated per J in a shared-memory hash table.
// Each G^D row lists a J once, so within one K only one thread updates J's slot, and the slots
// take their terms in ascending K (separately rounded FP64 products and sums): the values do not
// depend on scheduling.  COUNT: the number of J != I with P_IJ > tau; FILL: those (J, P_IJ).
constexpr int kTwoHopSlots = 2048;

template <bool FILL>
__global__ void twohop_kernel(const double* R, int N, CellGrid g, const long long* nptr, const int* ncol,
                              const long long* gptr, const int* gcol, const double* gval, double alpha, double tau,
                              int* pcnt, const long long* pptr, int* pcol, double* pval, int* err) {
  __shared__ int key[kTwoHopSlots];
  __shared__ double acc[kTwoHopSlots];
  __shared__ int s_n, s_fail, s_pos;
  const int i = blockIdx.x;
  for (int t = threadIdx.x; t < kTwoHopSlots; t += blockDim.x) {
    key[t] = -1;
    acc[t] = 0.0;
  }
  const long long b = nptr[i];
  const int deg = (int)(nptr[i + 1] - b);
  if (threadIdx.x == 0) {
    s_n = 0;
    s_fail = 0;
    int pos = 0;                                   // I's place among its sorted neighbours
    while (pos < deg && ncol[b + pos] < i) ++pos;
    s_pos = pos;
  }
  __syncthreads();
  const int pos_i = s_pos;
  for (int m = 0; m <= deg; ++m) {
    int k;
    double w;
    if (m == pos_i) {
      k = i;
      w = 1.0;
    } else {
      k = ncol[b + (m < pos_i ? m : m - 1)];
      w = exp(__dmul_rn(-alpha, min_image_r2(R, i, k, g.box)));
    }
    for (long long p = gptr[k] + threadIdx.x; p < gptr[k + 1]; p += blockDim.x) {
      const int j = gcol[p];
      if (j < 0 || j >= N) continue;
      const double term = __dmul_rn(w, gval[p]);
      unsigned h = ((unsigned)j * 2654435761u) >> (32 - 11);
      int probes = 0;
      for (;;) {
        const int old = atomicCAS(&key[h], -1, j);
        if (old == -1 || old == j) {
          acc[h] = __dadd_rn(acc[h], term);
          break;
        }
        h = (h + 1) & (kTwoHopSlots - 1);
        if (++probes >= kTwoHopSlots) {
          s_fail = 1;
          break;
        }
      }
    }
    __syncthreads();
  }
  if (s_fail) {
    if (threadIdx.x == 0) {
      atomicOr(err, kErrCapacity);
      if (!FILL) pcnt[i] = 0;
    }
    return;
  }
  for (int t = threadIdx.x; t < kTwoHopSlots; t += blockDim.x) {
    const int j = key[t];
    if (j < 0 || j == i || !(acc[t] > tau)) continue;
    const int slot = atomicAdd(&s_n, 1);
    if (FILL && slot < (int)(pptr[i + 1] - pptr[i])) {   // the count pass sized the row
      pcol[pptr[i] + slot] = j;
      pval[pptr[i] + slot] = acc[t];
    }
  }
  __syncthreads();
  if (!FILL && threadIdx.x == 0) pcnt[i] = s_n;
}

// Exclusive scan of int counts into int64 offsets (single CTA, N up to a few 1e5).
__global__ void scan_kernel(const int* cnt, int N, long long* out) {
  __shared__ long long part[1024];
  const int per = (N + blockDim.x - 1) / blockDim.x;
  const int b = threadIdx.x * per, e = min(N, b + per);
  long long s = 0;
  for (int i = b; i < e; ++i) s += cnt[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long acc = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) { const long long v = part[t]; part[t] = acc; acc += v; }
    out[N] = acc;
  }
  __syncthreads();
  long long acc = part[threadIdx.x];
  for (int i = b; i < e; ++i) { out[i] = acc; acc += cnt[i]; }
}

// ---- recursive coordinate bisection ---------------------------------------------------------
// Each block sorts one segment of perm by (key, index) using a global scratch of length P2.
__device__ void block_bitonic(double* key, int* idx, int P2) {
  for (int k = 2; k <= P2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < P2; t += blockDim.x) {
        const int u = t ^ j;
        if (u > t) {
          const bool up = (t & k) == 0;
          const double ka = key[t], kb = key[u];
          const int ia = idx[t], ib = idx[u];
          const bool gt = (ka > kb) || (ka == kb && ia > ib);
          if (gt == up) { key[t] = kb; key[u] = ka; idx[t] = ib; idx[u] = ia; }
        }
      }
      __syncthreads();
    }
}

__global__ void rcb_level_kernel(const RcbSeg* segs, int* perm, const double* R, CellGrid g, double* skey, int* sidx,
                                 int sort_by_index) {
  const RcbSeg sg = segs[blockIdx.x];
  const int n = sg.count;
  int P2 = 1;
  while (P2 < n) P2 <<= 1;
  double* key = skey + sg.scratch;
  int* idx = sidx + sg.scratch;
  __shared__ double smin[3][32], smax[3][32];
  __shared__ int axis_s;
  if (!sort_by_index) {
    // min / max are exact, so the reduction order does not matter
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int a = perm[sg.start + t];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double w = wrap1(R[3 * a + d], g.box[d]);
        mn[d] = fmin(mn[d], w);
        mx[d] = fmax(mx[d], w);
      }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
      for (int o = 16; o > 0; o >>= 1) {
        mn[d] = fmin(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
        mx[d] = fmax(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
      }
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0)
      for (int d = 0; d < 3; ++d) { smin[d][wid] = mn[d]; smax[d][wid] = mx[d]; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double e[3];
      for (int d = 0; d < 3; ++d) {
        double lo = smin[d][0], hi = smax[d][0];
        for (int q = 1; q < nw; ++q) { lo = fmin(lo, smin[d][q]); hi = fmax(hi, smax[d][q]); }
        e[d] = __dsub_rn(hi, lo);
      }
      int ax = 0;
      double best = e[0];
      if (e[1] > best) { ax = 1; best = e[1]; }
      if (e[2] > best) { ax = 2; }
      axis_s = ax;
    }
    __syncthreads();
  }
  const int ax = sort_by_index ? 0 : axis_s;
  for (int t = threadIdx.x; t < P2; t += blockDim.x) {
    if (t < n) {
      const int a = perm[sg.start + t];
      key[t] = sort_by_index ? (double)a : wrap1(R[3 * a + ax], g.box[ax]);
      idx[t] = a;
    } else {
      key[t] = 1e308;
      idx[t] = 0x7fffffff;
    }
  }
  __syncthreads();
  block_bitonic(key, idx, P2);
  for (int t = threadIdx.x; t < n; t += blockDim.x) perm[sg.start + t] = idx[t];
}

// ---- halos ----------------------------------------------------------------------------------
__global__ void halo_mark_kernel(const long long* row_ptr, const int* col, const int* perm, const RcbSeg* leaves,
                                 unsigned* bits, int words) {
  const RcbSeg lf = leaves[blockIdx.x];
  unsigned* b = bits + (long long)blockIdx.x * words;
  for (int t = threadIdx.x; t < words; t += blockDim.x) b[t] = 0u;
  __syncthreads();
  for (int q = 0; q < lf.count; ++q) {
    const int a = perm[lf.start + q];
    for (long long p = row_ptr[a] + threadIdx.x; p < row_ptr[a + 1]; p += blockDim.x) {
      const int j = col[p];
      atomicOr(&b[j >> 5], 1u << (j & 31));
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < lf.count; q += blockDim.x) {
    const int a = perm[lf.start + q];
    atomicAnd(&b[a >> 5], ~(1u << (a & 31)));
  }
}

__global__ void halo_count_kernel(const unsigned* bits, int words, int* hcnt) {
  const unsigned* b = bits + (long long)blockIdx.x * words;
  int s = 0;
  for (int t = threadIdx.x; t < words; t += blockDim.x) s += __popc(b[t]);
  __shared__ int red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < (unsigned)o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) hcnt[blockIdx.x] = red[0];
}

// Write subgraph atom lists: core atoms (ascending) then halo atoms (ascending).
__global__ void sub_fill_kernel(const unsigned* bits, int words, const int* perm, const RcbSeg* leaves,
                                const long long* sub_ptr, int* sub_atoms) {
  const RcbSeg lf = leaves[blockIdx.x];
  const unsigned* b = bits + (long long)blockIdx.x * words;
  const long long base = sub_ptr[blockIdx.x];
  for (int q = threadIdx.x; q < lf.count; q += blockDim.x) sub_atoms[base + q] = perm[lf.start + q];
  // ordered compaction of the bitmap: one warp walks words in order
  if (threadIdx.x < 32) {
    long long pos = base + lf.count;
    for (int w0 = 0; w0 < words; w0 += 32) {
      const int wi = w0 + threadIdx.x;
      const unsigned v = (wi < words) ? b[wi] : 0u;
      const int c = __popc(v);
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)threadIdx.x >= o) incl += y;
      }
      long long p = pos + incl - c;
      unsigned vv = v;
      while (vv) {
        const int bit = __ffs(vv) - 1;
        sub_atoms[p++] = wi * 32 + bit;
        vv &= vv - 1;
      }
      pos += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

}  // namespace

// ===============================================================================================
GraphBuilder::~GraphBuilder() { release(); }

void GraphBuilder::release() {
  for (void* p : {(void*)cell_of, (void*)cell_count, (void*)cell_start, (void*)cell_fill, (void*)cell_atoms,
                  (void*)cnt, (void*)fillc, (void*)ucnt, (void*)cptr, (void*)cand, (void*)n_cnt, (void*)n_ptr,
                  (void*)n_col, (void*)p_cnt, (void*)p_ptr, (void*)p_col, (void*)p_val})
    if (p) cudaFree(p);
  cell_of = cell_count = cell_start = cell_fill = cell_atoms = cnt = fillc = ucnt = nullptr;
  cptr = nullptr;
  cand = nullptr;
  n_cnt = p_cnt = n_col = p_col = nullptr;
  n_ptr = p_ptr = nullptr;
  p_val = nullptr;
  cap_n = cap_cells = 0;
  cap_cand = cap_ncol = cap_p = 0;
}

static CellGrid make_grid(const double box[3], double rc, int exact = 1) {
  CellGrid g;
  g.brute = 0;
  g.exact = exact;
  for (int a = 0; a < 3; ++a) {
    g.box[a] = box[a];
    g.nc[a] = (int)floor(box[a] / (rc * (1.0 + 1e-9) + 1e-9));
    if (g.nc[a] < 3) g.brute = 1;
    g.nc[a] = g.nc[a] < 1 ? 1 : g.nc[a];
    g.cw[a] = box[a] / g.nc[a];
  }
  return g;
}

cudaError_t GraphBuilder::build(const double* dR, int N, const double box[3], double r_graph, const long long* gptr,
                                const int* gcol, const double* gval, double tau, long long* row_ptr, int** col_out,
                                long long* col_cap, long long* nnz_host, int* derr, cudaStream_t s, bool exact,
                                bool keep_prev, int rule, double alpha) {
  cudaError_t e;
  const bool two_hop = rule == 1 && gptr != nullptr;
  const double rn2 = two_hop ? std::log(2.0 / tau) / alpha : 0.0;   // G^N neighbour list: R^2 < rn2
  CellGrid g = make_grid(box, two_hop ? std::sqrt(rn2) : r_graph, exact ? 1 : 0);
  const int ncell = g.nc[0] * g.nc[1] * g.nc[2];
  if (N > cap_n) {
    for (int** p : {&cell_of, &cnt, &fillc, &ucnt}) { if (*p) cudaFree(*p); *p = nullptr; }
    if (cptr) cudaFree(cptr);
    if ((e = cudaMalloc(&cell_of, sizeof(int) * N))) return e;
    if ((e = cudaMalloc(&cnt, sizeof(int) * N))) return e;
    if ((e = cudaMalloc(&fillc, sizeof(int) * N))) return e;
    if ((e = cudaMalloc(&ucnt, sizeof(int) * N))) return e;
    if ((e = cudaMalloc(&cptr, sizeof(long long) * (N + 1)))) return e;
    if (cell_atoms) cudaFree(cell_atoms);
    if ((e = cudaMalloc(&cell_atoms, sizeof(int) * N))) return e;
    for (int** p : {&n_cnt, &p_cnt}) { if (*p) cudaFree(*p); *p = nullptr; }
    for (long long** p : {&n_ptr, &p_ptr}) { if (*p) cudaFree(*p); *p = nullptr; }
    if ((e = cudaMalloc(&n_cnt, sizeof(int) * N))) return e;
    if ((e = cudaMalloc(&p_cnt, sizeof(int) * N))) return e;
    if ((e = cudaMalloc(&n_ptr, sizeof(long long) * (N + 1)))) return e;
    if ((e = cudaMalloc(&p_ptr, sizeof(long long) * (N + 1)))) return e;
    cap_n = N;
  }
  if (ncell > cap_cells) {
    for (int** p : {&cell_count, &cell_start, &cell_fill}) { if (*p) cudaFree(*p); *p = nullptr; }
    if ((e = cudaMalloc(&cell_count, sizeof(int) * ncell))) return e;
    if ((e = cudaMalloc(&cell_start, sizeof(int) * (ncell + 1)))) return e;
    if ((e = cudaMalloc(&cell_fill, sizeof(int) * ncell))) return e;
    cap_cells = ncell;
  }
  const int TB = 128, nb = (N + TB - 1) / TB;
  const double rg2 = r_graph * r_graph;
  if (!g.brute) {
    cudaMemsetAsync(cell_count, 0, sizeof(int) * ncell, s);
    cudaMemsetAsync(cell_fill, 0, sizeof(int) * ncell, s);
    cell_assign_kernel<<<nb, TB, 0, s>>>(dR, N, g, cell_of, cell_count);
    cell_scan_kernel<<<1, 1024, 0, s>>>(cell_count, ncell, cell_start);
    cell_fill_kernel<<<nb, TB, 0, s>>>(cell_of, N, cell_start, cell_fill, cell_atoms);
  }
  const int nbw = (N + 3) / 4;   // warp per atom, four per block
  if (two_hop) {
    // G^N rows: the neighbour list within rn2, each row sorted ascending
    count_dist_kernel<<<nbw, 128, 0, s>>>(dR, N, g, cell_of, cell_start, cell_count, cell_atoms, rn2, n_cnt);
    scan_kernel<<<1, 1024, 0, s>>>(n_cnt, N, n_ptr);
    long long nn = 0;
    cudaMemcpyAsync(&nn, n_ptr + N, sizeof(long long), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) return e;
    if (nn > cap_ncol) {
      if (n_col) cudaFree(n_col);
      cap_ncol = nn + nn / 4 + 1024;
      if ((e = cudaMalloc(&n_col, sizeof(int) * cap_ncol))) return e;
    }
    fill_dist_kernel<<<nbw, 128, 0, s>>>(dR, N, g, cell_of, cell_start, cell_count, cell_atoms, rn2, n_ptr, fillc,
                                         n_col);
    row_unique_kernel<<<N, 256, 8192 * sizeof(int), s>>>(n_ptr, n_col, ucnt, derr, 8192);
    // P = G^N G^D above tau, row by row (count, then fill)
    twohop_kernel<false><<<N, 256, 0, s>>>(dR, N, g, n_ptr, n_col, gptr, gcol, gval, alpha, tau, p_cnt, nullptr,
                                           nullptr, nullptr, derr);
    scan_kernel<<<1, 1024, 0, s>>>(p_cnt, N, p_ptr);
    long long np = 0;
    cudaMemcpyAsync(&np, p_ptr + N, sizeof(long long), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) return e;
    if (np > cap_p) {
      if (p_col) cudaFree(p_col);
      if (p_val) cudaFree(p_val);
      cap_p = np + np / 4 + 1024;
      if ((e = cudaMalloc(&p_col, sizeof(int) * cap_p))) return e;
      if ((e = cudaMalloc(&p_val, sizeof(double) * cap_p))) return e;
    }
    twohop_kernel<true><<<N, 256, 0, s>>>(dR, N, g, n_ptr, n_col, gptr, gcol, gval, alpha, tau, nullptr, p_ptr,
                                          p_col, p_val, derr);
    // the entries of P above tau are the rule's edges, added in both directions
    cudaMemsetAsync(cnt, 0, sizeof(int) * N, s);
    count_gd_kernel<<<N, 64, 0, s>>>(p_ptr, p_col, p_val, N, tau, cnt);
  } else {
    count_dist_kernel<<<nbw, 128, 0, s>>>(dR, N, g, cell_of, cell_start, cell_count, cell_atoms, rg2, cnt);
    if (gptr) count_gd_kernel<<<N, 64, 0, s>>>(gptr, gcol, gval, N, tau, cnt);
  }
  // keep_prev: the edges of the graph currently in row_ptr / col_out are candidates as well (they
  // are read here, before the new graph overwrites them)
  if (keep_prev) count_prev_kernel<<<nb, TB, 0, s>>>(row_ptr, N, cnt);
  scan_kernel<<<1, 1024, 0, s>>>(cnt, N, cptr);
  long long ncand = 0;
  cudaMemcpyAsync(&ncand, cptr + N, sizeof(long long), cudaMemcpyDeviceToHost, s);
  if ((e = cudaStreamSynchronize(s))) return e;
  if (ncand > cap_cand) {
    if (cand) cudaFree(cand);
    cap_cand = ncand + ncand / 4 + 1024;
    if ((e = cudaMalloc(&cand, sizeof(int) * cap_cand))) return e;
  }
  if (two_hop) {
    cudaMemsetAsync(fillc, 0, sizeof(int) * N, s);
    fill_gd_kernel<<<N, 64, 0, s>>>(p_ptr, p_col, p_val, N, tau, cptr, fillc, cand);
  } else {
    fill_dist_kernel<<<nbw, 128, 0, s>>>(dR, N, g, cell_of, cell_start, cell_count, cell_atoms, rg2, cptr, fillc,
                                         cand);
    if (gptr) fill_gd_kernel<<<N, 64, 0, s>>>(gptr, gcol, gval, N, tau, cptr, fillc, cand);
  }
  if (keep_prev) fill_prev_kernel<<<N, 64, 0, s>>>(row_ptr, *col_out, N, cptr, fillc, cand);
  const int cap = 8192;
  row_unique_kernel<<<N, 256, cap * sizeof(int), s>>>(cptr, cand, ucnt, derr, cap);
  scan_kernel<<<1, 1024, 0, s>>>(ucnt, N, row_ptr);
  long long nnz = 0;
  cudaMemcpyAsync(&nnz, row_ptr + N, sizeof(long long), cudaMemcpyDeviceToHost, s);
  if ((e = cudaStreamSynchronize(s))) return e;
  if (nnz > *col_cap) {
    if (*col_out) cudaFree(*col_out);
    *col_cap = nnz + nnz / 4 + 1024;
    if ((e = cudaMalloc(col_out, sizeof(int) * (*col_cap)))) return e;
  }
  compact_kernel<<<N, 128, 0, s>>>(cptr, cand, row_ptr, N, *col_out);
  *nnz_host = nnz;
  return cudaGetLastError();
}

// ===============================================================================================
Partitioner::~Partitioner() { release(); }

void Partitioner::release() {
  for (void* p : {(void*)perm, (void*)skey, (void*)sidx, (void*)segs_d, (void*)bits, (void*)hcnt})
    if (p) cudaFree(p);
  perm = nullptr; skey = nullptr; sidx = nullptr; segs_d = nullptr; bits = nullptr; hcnt = nullptr;
  cap_n = cap_scr = cap_seg = 0;
  cap_hcnt = cap_subptr = 0;
  cap_bits = 0;
}

static int next_pow2(int n) { int p = 1; while (p < n) p <<= 1; return p; }

cudaError_t Partitioner::rcb(const double* dR, int N, const double box[3], int core_size, cudaStream_t s) {
  cudaError_t e;
  n_parts = N / core_size;
  {
    const double q = (double)N / core_size;
    n_parts = (int)rint(q);
    if (n_parts < 1) n_parts = 1;
  }
  if (N > cap_n) {
    if (perm) cudaFree(perm);
    if ((e = cudaMalloc(&perm, sizeof(int) * N))) return e;
    cap_n = N;
  }
  const long long need_scr = 2LL * next_pow2(N) + 64;
  if (need_scr > cap_scr) {
    if (skey) cudaFree(skey);
    if (sidx) cudaFree(sidx);
    if ((e = cudaMalloc(&skey, sizeof(double) * need_scr))) return e;
    if ((e = cudaMalloc(&sidx, sizeof(int) * need_scr))) return e;
    cap_scr = need_scr;
  }
  if (n_parts + 1 > cap_seg) {
    if (segs_d) cudaFree(segs_d);
    if ((e = cudaMalloc(&segs_d, sizeof(RcbSeg) * (n_parts + 1)))) return e;
    cap_seg = n_parts + 1;
  }
  std::vector<int> hp(N);
  for (int i = 0; i < N; ++i) hp[i] = i;
  cudaMemcpyAsync(perm, hp.data(), sizeof(int) * N, cudaMemcpyHostToDevice, s);
  CellGrid g = make_grid(box, 1.0);
  struct Node { int start, count, p; };
  std::vector<Node> level = {{0, N, n_parts}};
  std::vector<RcbSeg> hs;
  while (true) {
    hs.clear();
    std::vector<Node> next;
    long long scr = 0;
    for (const Node& nd : level) {
      if (nd.p == 1) { next.push_back(nd); continue; }
      RcbSeg sg;
      sg.start = nd.start; sg.count = nd.count; sg.scratch = scr;
      scr += next_pow2(nd.count);
      hs.push_back(sg);
      const int pl = nd.p / 2;
      const int m = (int)(((long long)nd.count * pl) / nd.p);
      next.push_back({nd.start, m, pl});
      next.push_back({nd.start + m, nd.count - m, nd.p - pl});
    }
    if (hs.empty()) break;
    cudaMemcpyAsync(segs_d, hs.data(), sizeof(RcbSeg) * hs.size(), cudaMemcpyHostToDevice, s);
    rcb_level_kernel<<<(int)hs.size(), 1024, 0, s>>>(segs_d, perm, dR, g, skey, sidx, 0);
    // the segment array is rewritten next level: wait before reuse
    if ((e = cudaStreamSynchronize(s))) return e;
    level = next;
  }
  // leaves in depth-first order: the level list is already in tree order
  leaves.clear();
  for (const Node& nd : level) leaves.push_back({nd.start, nd.count, 0});
  // sort every leaf by atom index
  long long scr = 0;
  for (auto& lf : leaves) { lf.scratch = scr; scr += next_pow2(lf.count); }
  if (scr > cap_scr) return cudaErrorMemoryAllocation;
  cudaMemcpyAsync(segs_d, leaves.data(), sizeof(RcbSeg) * leaves.size(), cudaMemcpyHostToDevice, s);
  rcb_level_kernel<<<(int)leaves.size(), 256, 0, s>>>(segs_d, perm, dR, g, skey, sidx, 1);
  return cudaStreamSynchronize(s);
}

cudaError_t Partitioner::set_cores(const std::vector<std::vector<int>>& cores, int N, cudaStream_t s) {
  cudaError_t e;
  if (N > cap_n) {
    if (perm) cudaFree(perm);
    if ((e = cudaMalloc(&perm, sizeof(int) * N))) return e;
    cap_n = N;
  }
  n_parts = (int)cores.size();
  if (n_parts + 1 > cap_seg) {
    if (segs_d) cudaFree(segs_d);
    if ((e = cudaMalloc(&segs_d, sizeof(RcbSeg) * (n_parts + 1)))) return e;
    cap_seg = n_parts + 1;
  }
  std::vector<int> hp;
  leaves.clear();
  for (auto& c : cores) {
    leaves.push_back({(int)hp.size(), (int)c.size(), 0});
    hp.insert(hp.end(), c.begin(), c.end());
  }
  if ((int)hp.size() > cap_n) return cudaErrorInvalidValue;
  cudaMemcpyAsync(perm, hp.data(), sizeof(int) * hp.size(), cudaMemcpyHostToDevice, s);
  return cudaStreamSynchronize(s);
}

cudaError_t Partitioner::halos(const long long* row_ptr, const int* col, int N, long long** sub_ptr_d, int** sub_atoms_d,
                               long long* sub_cap, std::vector<long long>& sub_ptr_h, cudaStream_t s) {
  cudaError_t e;
  const int words = (N + 31) / 32;
  const long long need = (long long)words * n_parts;
  if (need > cap_bits) {
    if (bits) cudaFree(bits);
    if ((e = cudaMalloc(&bits, sizeof(unsigned) * need))) return e;
    cap_bits = need;
  }
  if (n_parts > cap_hcnt) {
    if (hcnt) cudaFree(hcnt);
    hcnt = nullptr;
    if ((e = cudaMalloc(&hcnt, sizeof(int) * n_parts))) return e;
    cap_hcnt = n_parts;
  }
  cudaMemcpyAsync(segs_d, leaves.data(), sizeof(RcbSeg) * leaves.size(), cudaMemcpyHostToDevice, s);
  halo_mark_kernel<<<n_parts, 256, 0, s>>>(row_ptr, col, perm, segs_d, bits, words);
  halo_count_kernel<<<n_parts, 256, 0, s>>>(bits, words, hcnt);
  std::vector<int> hh(n_parts);
  cudaMemcpyAsync(hh.data(), hcnt, sizeof(int) * n_parts, cudaMemcpyDeviceToHost, s);
  if ((e = cudaStreamSynchronize(s))) return e;
  halo_count_h = hh;
  sub_ptr_h.assign(n_parts + 1, 0);
  for (int i = 0; i < n_parts; ++i) sub_ptr_h[i + 1] = sub_ptr_h[i] + leaves[i].count + hh[i];
  const long long tot = sub_ptr_h[n_parts];
  if (tot > *sub_cap) {
    if (*sub_atoms_d) cudaFree(*sub_atoms_d);
    *sub_cap = tot + tot / 4 + 1024;
    if ((e = cudaMalloc(sub_atoms_d, sizeof(int) * (*sub_cap)))) return e;
  }
  if (n_parts + 1 > cap_subptr) {
    if (*sub_ptr_d) cudaFree(*sub_ptr_d);
    *sub_ptr_d = nullptr;
    if ((e = cudaMalloc(sub_ptr_d, sizeof(long long) * (n_parts + 1)))) return e;
    cap_subptr = n_parts + 1;
  }
  cudaMemcpyAsync(*sub_ptr_d, sub_ptr_h.data(), sizeof(long long) * (n_parts + 1), cudaMemcpyHostToDevice, s);
  sub_fill_kernel<<<n_parts, 128, 0, s>>>(bits, words, perm, segs_d, *sub_ptr_d, *sub_atoms_d);
  return cudaStreamSynchronize(s);
}

}  // namespace sedacs
