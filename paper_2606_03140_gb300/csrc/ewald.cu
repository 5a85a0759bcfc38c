// Periodic Gaussian-gamma Coulomb potential V = gamma b and the gradient of a^T gamma b
// by Ewald summation (SCC-DFTB screened Coulomb, SI Sec. D; GPU Ewald, Sec. "Scalability").
//
//   gamma_IJ = sum_L' [erfc(eta d) - erfc(a_IJ d)] / d
//            + (4 pi / V) sum_{k != 0} exp(-k^2/4eta^2)/k^2 cos(k.(R_J - R_I))
//            - pi / (eta^2 V) + delta_IJ (U_I - 2 eta / sqrt(pi)),
//   a_IJ = 1 / sqrt(2 (sigma_I^2 + sigma_J^2)),  sigma_I = 1 / (sqrt(pi) U_I).
//
// Reciprocal space uses separable phase tables: e^{ik.R} = X[m1] Y[m2] Z[m3] with
// X[m] = exp(2 pi i m x / L).  k-vectors are grouped in rows of fixed (m1, m2); one CTA
// accumulates a row's structure factor over a chunk of atoms (products X*Y once per atom
// in shared memory, the Z table row read coalesced), partial sums are reduced in FP64 in a
// fixed order.  The potential kernel keeps each atom's Z row in shared memory and streams
// the k-rows.  T = float for the mixed path (FP64 final sums), double for the plain path.
#include <cmath>
#include <mutex>
#include <vector>
#include "ewald.cuh"

namespace sedacs {

namespace {

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

template <typename T>
__device__ __forceinline__ typename C2<T>::t cmul(typename C2<T>::t a, typename C2<T>::t b) {
  typename C2<T>::t r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// Phase tables in FP64, stored as T: tab[(axis * N + J) * (nmax + 1) + m] = exp(2 pi i m u), u = x / L.
template <typename T>
__global__ void phase_table_kernel(const double* R, int N, EwaldGeom g, typename C2<T>::t* tab) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= N) return;
  for (int a = 0; a < 3; ++a) {
    const double u = R[3 * J + a] / g.box_b[a] / kBohrA * 1.0;   // x (A) -> bohr -> fraction
    double s, c;
    sincospi(2.0 * (u - floor(u)), &s, &c);
    double re = 1.0, im = 0.0;
    const int nm = g.nmax[a];
    typename C2<T>::t* row = tab + ((long long)a * N + J) * (g.nmax_all + 1);
    for (int m = 0; m <= nm; ++m) {
      row[m].x = (T)re;
      row[m].y = (T)im;
      const double nr = re * c - im * s, ni = re * s + im * c;
      re = nr;
      im = ni;
    }
  }
}

// S_row[m3] partial over an atom chunk, for nvec charge vectors.
template <typename T, int NV>
__global__ void structure_factor_kernel(const KRow* rows, const typename C2<T>::t* tab, const double* b0,
                                        const double* b1, int N, int nmax_all, int chunk, double* part,
                                        long long nk_total) {
  using CT = typename C2<T>::t;
  const KRow kr = rows[blockIdx.x];
  const int a0 = blockIdx.y * chunk;
  const int a1 = min(N, a0 + chunk);
  extern __shared__ unsigned char sm[];
  CT* c12 = reinterpret_cast<CT*>(sm);   // [chunk][NV]
  for (int J = a0 + threadIdx.x; J < a1; J += blockDim.x) {
    CT x = tab[(0LL * N + J) * (nmax_all + 1) + kr.m1];
    const int am2 = abs(kr.m2);
    CT y = tab[(1LL * N + J) * (nmax_all + 1) + am2];
    if (kr.m2 < 0) y.y = -y.y;
    const CT xy = cmul<T>(x, y);
    CT v0;
    v0.x = (T)b0[J] * xy.x;
    v0.y = (T)b0[J] * xy.y;
    c12[(J - a0) * NV] = v0;
    if (NV > 1) {
      CT v1;
      v1.x = (T)b1[J] * xy.x;
      v1.y = (T)b1[J] * xy.y;
      c12[(J - a0) * NV + 1] = v1;
    }
  }
  __syncthreads();
  // 4 groups of 64 threads: lane = m3 slot, group = every 4th atom of the chunk; the group
  // partials are added in a fixed order through shared memory.
  const int nm3 = kr.m3hi - kr.m3lo + 1;
  const int grp = threadIdx.x >> 6, ln = threadIdx.x & 63;
  T* red = reinterpret_cast<T*>(c12 + (size_t)chunk * NV);   // [4][64][NV][2] after the products
  for (int base = 0; base < nm3; base += 64) {      // block-uniform loop over 64 m3 slots at a time
    T sr[NV], si[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) { sr[v] = 0; si[v] = 0; }
    const int t = base + ln;
    const int m3 = kr.m3lo + t;
    const int am3 = abs(m3);
    if (t < nm3) {
      for (int J = a0 + grp; J < a1; J += 4) {
        CT z = tab[(2LL * N + J) * (nmax_all + 1) + am3];
        if (m3 < 0) z.y = -z.y;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const CT c = c12[(J - a0) * NV + v];
          sr[v] += c.x * z.x - c.y * z.y;
          si[v] += c.x * z.y + c.y * z.x;
        }
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      red[((grp * 64 + ln) * NV + v) * 2] = sr[v];
      red[((grp * 64 + ln) * NV + v) * 2 + 1] = si[v];
    }
    __syncthreads();
    if (grp == 0 && t < nm3) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double re = 0.0, im = 0.0;
        for (int g2 = 0; g2 < 4; ++g2) {
          re += (double)red[((g2 * 64 + ln) * NV + v) * 2];
          im += (double)red[((g2 * 64 + ln) * NV + v) * 2 + 1];
        }
        const long long o = ((long long)blockIdx.y * NV + v) * nk_total + kr.koff + t;
        part[2 * o] = re;
        part[2 * o + 1] = im;
      }
    }
    __syncthreads();
  }
}

// S(k) = sum over atom chunks (fixed order), times the k weight; stored as T complex.
template <typename T>
__global__ void sf_reduce_kernel(const double* part, int nchunk, int nv, long long nk, const double* wk,
                                 typename C2<T>::t* ws) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= nk) return;
  for (int v = 0; v < nv; ++v) {
    double re = 0.0, im = 0.0;
    for (int c = 0; c < nchunk; ++c) {
      const long long o = ((long long)c * nv + v) * nk + k;
      re += part[2 * o];
      im += part[2 * o + 1];
    }
    ws[v * nk + k].x = (T)(wk[k] * re);
    ws[v * nk + k].y = (T)(wk[k] * im);
  }
}

// Per atom I: sum_k w S(k) e^{-ik.R_I} -> Re (potential) and, for gradients, Im weighted by k.
// mode 0: out[I] = Re sum (nv = 1).  mode 1: g[I][c] = sum w k_c [a_I Im(S_b e^-ikR) + b_I Im(S_a e^-ikR)].
template <typename T, int MODE>
__global__ void recip_atom_kernel(const KRow* rows, int nrows, const typename C2<T>::t* tab, const typename C2<T>::t* ws,
                                  long long nk, int N, int nmax_all, int m3max, EwaldGeom g, const double* av,
                                  const double* bv, double* out_part) {
  // block (atom chunk, row chunk): rows [r0, r1) of the k list, partial sums per row chunk
  const int rchunk = (nrows + gridDim.y - 1) / gridDim.y;
  const int r0 = blockIdx.y * rchunk, r1 = min(nrows, r0 + rchunk);
  double* out = out_part + (long long)blockIdx.y * (MODE == 0 ? N : 3 * N);
  using CT = typename C2<T>::t;
  extern __shared__ unsigned char sm[];
  CT* zt = reinterpret_cast<CT*>(sm);          // [blockDim][2*m3max+1]
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int W = 2 * m3max + 1;
  CT* myz = zt + threadIdx.x * W;
  if (I < N) {
    for (int m = 0; m <= m3max; ++m) {
      const CT z = tab[(2LL * N + I) * (nmax_all + 1) + m];
      CT zc = z;
      zc.y = -zc.y;
      myz[m3max + m] = zc;           // conj(Z[m]) for e^{-ik.R}
      CT zp = z;
      myz[m3max - m] = zp;           // conj(Z[-m]) = Z[m]
    }
  }
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
  const double tpx = 2.0 * M_PI / g.box_b[0], tpy = 2.0 * M_PI / g.box_b[1], tpz = 2.0 * M_PI / g.box_b[2];
  if (I < N) {
    for (int r = r0; r < r1; ++r) {
      const KRow kr = rows[r];
      CT x = tab[(0LL * N + I) * (nmax_all + 1) + kr.m1];
      CT y = tab[(1LL * N + I) * (nmax_all + 1) + abs(kr.m2)];
      if (kr.m2 < 0) y.y = -y.y;
      CT xy = cmul<T>(x, y);
      xy.y = -xy.y;                     // conj -> e^{-i(k1 x + k2 y)}
      const int nm3 = kr.m3hi - kr.m3lo + 1;
      if (MODE == 0) {
        T re = 0;
        for (int t = 0; t < nm3; ++t) {
          const CT s = ws[kr.koff + t];
          const CT z = myz[m3max + kr.m3lo + t];
          const CT e = cmul<T>(xy, z);
          re += s.x * e.x - s.y * e.y;
        }
        acc0 += (double)re;
      } else {
        // Im(S e^{-ikR}) for S_b (vector 0) and S_a (vector 1)
        T i1 = 0, i3 = 0;   // sums over m3 of the Im-combination weighted by 1 and by m3
        for (int t = 0; t < nm3; ++t) {
          const int m3 = kr.m3lo + t;
          const CT sb = ws[kr.koff + t];
          const CT sa = ws[nk + kr.koff + t];
          const CT z = myz[m3max + m3];
          const CT e = cmul<T>(xy, z);
          const T imb = sb.x * e.y + sb.y * e.x;
          const T ima = sa.x * e.y + sa.y * e.x;
          const T comb = (T)av[I] * imb + (T)bv[I] * ima;
          i1 += comb;
          i3 += comb * (T)m3;
        }
        acc0 += (double)i1 * (tpx * kr.m1);
        acc1 += (double)i1 * (tpy * kr.m2);
        acc2 += (double)i3 * tpz;
      }
    }
    if (MODE == 0) out[I] = acc0;
    else {
      out[3 * I] = acc0;
      out[3 * I + 1] = acc1;
      out[3 * I + 2] = acc2;
    }
  }
}

// Real-space part, one warp per atom I over images within rc.  mode 0: V_I += sum_J phi b_J;
// mode 1: dE/dR_I += -sum_J (a_I b_J + a_J b_I) phi'(d) d_hat.  Differences of positions are
// taken in FP64, the rest in T; lane sums are combined by a fixed shuffle tree.
template <typename T, int MODE>
__global__ void real_space_kernel(const double* R, const int* species, int N, EwaldGeom g, const int* cell_start,
                                  const int* cell_count, const int* cell_atoms, const int* cell_of, const double* av,
                                  const double* bv, double* out) {
  const int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (I >= N) return;
  const T rc2 = (T)(g.rc_b * g.rc_b);
  const T eta = (T)g.eta;
  const T sq = (T)1.1283791670955126;    // 2 / sqrt(pi)
  const T inv_b = (T)(1.0 / kBohrA);
  const T bx = (T)g.box_b[0], by = (T)g.box_b[1], bz = (T)g.box_b[2];
  const int si = species[I];
  double acc = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
  const double xi = R[3 * I], yi = R[3 * I + 1], zi = R[3 * I + 2];
  auto visit = [&](int J, T dx, T dy, T dz) {
    const T d2 = dx * dx + dy * dy + dz * dz;
    if (d2 >= rc2 || d2 == (T)0) return;
    const T d = sqrt(d2);
    const T aij = (T)g.a[si][species[J]];
    const T e1 = erfc(eta * d), e2 = erfc(aij * d);
    const T phi = (e1 - e2) / d;
    if (MODE == 0) {
      acc += (double)phi * bv[J];
    } else {
      const T dphi = (-sq * eta * exp(-(eta * d) * (eta * d)) + sq * aij * exp(-(aij * d) * (aij * d))) / d - phi / d;
      const double coef = (av[I] * bv[J] + av[J] * bv[I]) * (double)(dphi / d);
      gx -= coef * (double)dx;
      gy -= coef * (double)dy;
      gz -= coef * (double)dz;
    }
  };
  auto rel = [&](int J, T& dx, T& dy, T& dz) {
    dx = (T)(R[3 * J] - xi) * inv_b;
    dy = (T)(R[3 * J + 1] - yi) * inv_b;
    dz = (T)(R[3 * J + 2] - zi) * inv_b;
    dx -= bx * rint(dx / bx);
    dy -= by * rint(dy / by);
    dz -= bz * rint(dz / bz);
  };
  if (g.brute) {
    for (int J = lane; J < N; J += 32) {
      T dx, dy, dz;
      rel(J, dx, dy, dz);
      for (int ix = -g.nimg[0]; ix <= g.nimg[0]; ++ix)
        for (int iy = -g.nimg[1]; iy <= g.nimg[1]; ++iy)
          for (int iz = -g.nimg[2]; iz <= g.nimg[2]; ++iz) visit(J, dx + ix * bx, dy + iy * by, dz + iz * bz);
    }
  } else {
    const int cid = cell_of[I];
    const int cz = cid % g.nc[2], cy = (cid / g.nc[2]) % g.nc[1], cx = cid / (g.nc[2] * g.nc[1]);
    for (int ddx = -1; ddx <= 1; ++ddx)
      for (int ddy = -1; ddy <= 1; ++ddy)
        for (int ddz = -1; ddz <= 1; ++ddz) {
          const int x = (cx + ddx + g.nc[0]) % g.nc[0];
          const int y = (cy + ddy + g.nc[1]) % g.nc[1];
          const int z = (cz + ddz + g.nc[2]) % g.nc[2];
          const int c = (x * g.nc[1] + y) * g.nc[2] + z;
          for (int q = lane; q < cell_count[c]; q += 32) {
            const int J = cell_atoms[cell_start[c] + q];
            T dx, dy, dz;
            rel(J, dx, dy, dz);
            visit(J, dx, dy, dz);
          }
        }
  }
  if (MODE == 0) {
    acc = warp_sum(acc);
    if (lane == 0) out[I] = acc;
  } else {
    gx = warp_sum(gx);
    gy = warp_sum(gy);
    gz = warp_sum(gz);
    if (lane == 0) {
      out[3 * I] = gx;
      out[3 * I + 1] = gy;
      out[3 * I + 2] = gz;
    }
  }
}

// ---- cell path of the real-space sum (cells at least rc wide, 3 or more per axis) -------------
// Atoms are ordered by cell, and by index inside a cell (deterministic).  Each sorted entry
// keeps its coordinates relative to its cell's origin (bohr) and its species; the warp of atom
// I scans the 27 neighbour cells with coalesced loads, queues the pairs inside rc in shared
// memory (ballot + popc) and evaluates them 32 at a time, so the erfc/exp work runs with
// full warps.

template <typename T> struct Pos4;
template <> struct Pos4<float> { using t = float4; };
template <> struct Pos4<double> { using t = double4; };

__global__ void cell_count_kernel(const double* R, int N, EwaldGeom g, int* cell_of, int* cell_count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int c[3];
  for (int a = 0; a < 3; ++a) {
    const double x = R[3 * i + a] / kBohrA;
    const double w = x - g.box_b[a] * floor(x / g.box_b[a]);
    c[a] = min(max((int)floor(w / (g.box_b[a] / g.nc[a])), 0), g.nc[a] - 1);
  }
  const int cid = (c[0] * g.nc[1] + c[1]) * g.nc[2] + c[2];
  cell_of[i] = cid;
  atomicAdd(&cell_count[cid], 1);
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

// block per cell: stable compaction of the atoms of the cell in index order, with their
// cell-relative coordinates
template <typename T>
__global__ void cell_fill_sorted_kernel(const double* R, const int* species, int N, EwaldGeom g, const int* cell_of,
                                        const int* cell_start, int* sorted_atom, typename Pos4<T>::t* pos_s) {
  const int c = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __shared__ int wcnt[32];
  __shared__ int base_sh;
  if (threadIdx.x == 0) base_sh = cell_start[c];
  const int cz = c % g.nc[2], cy = (c / g.nc[2]) % g.nc[1], cx = c / (g.nc[2] * g.nc[1]);
  const double o[3] = {cx * (g.box_b[0] / g.nc[0]), cy * (g.box_b[1] / g.nc[1]), cz * (g.box_b[2] / g.nc[2])};
  __syncthreads();
  for (int i0 = 0; i0 < N; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    const bool mine = i < N && cell_of[i] == c;
    const unsigned m = __ballot_sync(0xffffffffu, mine);
    if (lane == 0) wcnt[warp] = __popc(m);
    __syncthreads();
    int off = 0;
    for (int w = 0; w < warp; ++w) off += wcnt[w];
    if (mine) {
      const int k = base_sh + off + __popc(m & ((1u << lane) - 1u));
      sorted_atom[k] = i;
      typename Pos4<T>::t p;
      double r[3];
      for (int a = 0; a < 3; ++a) {
        const double x = R[3 * i + a] / kBohrA;
        r[a] = (x - g.box_b[a] * floor(x / g.box_b[a])) - o[a];
      }
      p.x = (T)r[0];
      p.y = (T)r[1];
      p.z = (T)r[2];
      p.w = (T)species[i];
      pos_s[k] = p;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < nw; ++w) tot += wcnt[w];
      base_sh += tot;
    }
    __syncthreads();
  }
}

template <typename T, int MODE>
__global__ void real_cells_kernel(const typename Pos4<T>::t* pos_s, const int* sorted_atom, const int* cell_start,
                                  int N, EwaldGeom g, const double* av, const double* bv, double* out) {
  constexpr int kQ = 64;
  __shared__ int qj[4][kQ];
  __shared__ T qd[4][kQ][3];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * 4 + wib;              // sorted index of atom I
  if (k >= N) return;
  const int I = sorted_atom[k];
  const typename Pos4<T>::t pi = pos_s[k];
  const int si = (int)pi.w;
  // cell of k: the one whose range holds k
  int lo = 0, hi = g.nc[0] * g.nc[1] * g.nc[2];
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (cell_start[mid] <= k) lo = mid; else hi = mid;
  }
  const int c = lo;
  const int cz = c % g.nc[2], cy = (c / g.nc[2]) % g.nc[1], cx = c / (g.nc[2] * g.nc[1]);
  const T wx = (T)(g.box_b[0] / g.nc[0]), wy = (T)(g.box_b[1] / g.nc[1]), wz = (T)(g.box_b[2] / g.nc[2]);
  const T rc2 = (T)(g.rc_b * g.rc_b);
  const T eta = (T)g.eta;
  const T sq = (T)1.1283791670955126;    // 2 / sqrt(pi)
  const double aI = MODE == 1 ? av[I] : 0.0, bI = MODE == 1 ? bv[I] : 0.0;
  double acc = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
  int qn = 0;
  auto flush = [&](int cnt) {
    // lanes < cnt take one queued pair each
    if (lane < cnt) {
      const int j = qj[wib][lane];
      const T dx = qd[wib][lane][0], dy = qd[wib][lane][1], dz = qd[wib][lane][2];
      const T d2 = dx * dx + dy * dy + dz * dz;
      const T d = sqrt(d2);
      const int sj = (int)pos_s[j].w;
      const int J = sorted_atom[j];
      const T aij = (T)g.a[si][sj];
      const T e1 = erfc(eta * d), e2 = erfc(aij * d);
      const T phi = (e1 - e2) / d;
      if (MODE == 0) {
        acc += (double)phi * bv[J];
      } else {
        const T dphi = (-sq * eta * exp(-(eta * d) * (eta * d)) + sq * aij * exp(-(aij * d) * (aij * d))) / d - phi / d;
        const double coef = (aI * bv[J] + av[J] * bI) * (double)(dphi / d);
        gx -= coef * (double)dx;
        gy -= coef * (double)dy;
        gz -= coef * (double)dz;
      }
    }
  };
  for (int ddx = -1; ddx <= 1; ++ddx)
    for (int ddy = -1; ddy <= 1; ++ddy)
      for (int ddz = -1; ddz <= 1; ++ddz) {
        const int x = (cx + ddx + g.nc[0]) % g.nc[0];
        const int y = (cy + ddy + g.nc[1]) % g.nc[1];
        const int z = (cz + ddz + g.nc[2]) % g.nc[2];
        const int cn = (x * g.nc[1] + y) * g.nc[2] + z;
        const int j0 = cell_start[cn], j1 = cell_start[cn + 1];
        const T ox = (T)ddx * wx - pi.x, oy = (T)ddy * wy - pi.y, oz = (T)ddz * wz - pi.z;
        for (int jb = j0; jb < j1; jb += 32) {
          const int j = jb + lane;
          bool in = false;
          T dx = 0, dy = 0, dz = 0;
          if (j < j1) {
            const typename Pos4<T>::t pj = pos_s[j];
            dx = pj.x + ox;
            dy = pj.y + oy;
            dz = pj.z + oz;
            const T d2 = dx * dx + dy * dy + dz * dz;
            in = d2 < rc2 && j != k;
          }
          const unsigned m = __ballot_sync(0xffffffffu, in);
          if (in) {
            const int slot = qn + __popc(m & ((1u << lane) - 1u));
            qj[wib][slot] = j;
            qd[wib][slot][0] = dx;
            qd[wib][slot][1] = dy;
            qd[wib][slot][2] = dz;
          }
          qn += __popc(m);
          __syncwarp();
          if (qn >= 32) {
            flush(32);
            __syncwarp();
            int tj = 0;
            T t0 = 0, t1 = 0, t2 = 0;
            if (lane < qn - 32) {
              tj = qj[wib][32 + lane];
              t0 = qd[wib][32 + lane][0];
              t1 = qd[wib][32 + lane][1];
              t2 = qd[wib][32 + lane][2];
            }
            __syncwarp();
            if (lane < qn - 32) {
              qj[wib][lane] = tj;
              qd[wib][lane][0] = t0;
              qd[wib][lane][1] = t1;
              qd[wib][lane][2] = t2;
            }
            qn -= 32;
            __syncwarp();
          }
        }
      }
  flush(qn);
  if (MODE == 0) {
    acc = warp_sum(acc);
    if (lane == 0) out[I] = acc;
  } else {
    gx = warp_sum(gx);
    gy = warp_sum(gy);
    gz = warp_sum(gz);
    if (lane == 0) {
      out[3 * I] = gx;
      out[3 * I + 1] = gy;
      out[3 * I + 2] = gz;
    }
  }
}

__global__ void chunk_reduce_kernel(const double* part, int nchunk, long long len, double* out) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= len) return;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[c * len + t];
  out[t] = s;
}

// out = real + recip + self/background terms (potential) or real + recip (gradient, Ha/A).
__global__ void combine_pot_kernel(const double* real, const double* recip, const double* b, const int* species,
                                   EwaldGeom g, const double* bsum, double* V, int N) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= N) return;
  V[I] = real[I] + recip[I] - M_PI / (g.eta * g.eta * g.vol) * bsum[0] +
         (g.u[species[I]] - 2.0 * g.eta / sqrt(M_PI)) * b[I];
}

__global__ void combine_grad_kernel(const double* real, const double* recip, double* G, int N, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * N) return;
  G[i] = (real[i] + recip[i]) * scale;
}

__global__ void sum_kernel(const double* b, int N, double* out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s += b[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

}  // namespace

// =================================================================================================
Ewald::~Ewald() { release(); }

void Ewald::release() {
  for (void* p : {(void*)rows_d, (void*)wk_d, (void*)tab, (void*)part, (void*)ws, (void*)real_buf, (void*)recip_buf,
                  (void*)cell_of, (void*)cell_count, (void*)cell_start, (void*)cell_atoms, (void*)scal, (void*)rpart,
                  pos_s})
    if (p) cudaFree(p);
  rows_d = nullptr; wk_d = nullptr; tab = nullptr; part = nullptr; ws = nullptr; real_buf = nullptr;
  recip_buf = nullptr; rpart = nullptr; cell_of = cell_count = cell_start = cell_atoms = nullptr; scal = nullptr;
  pos_s = nullptr;
  N_ = 0;
}

cudaError_t Ewald::setup(int N, const double box_A[3], const double hubbard_u[3], bool fp64, double tol) {
  release();
  N_ = N;
  fp64_ = fp64;
  const double x = sqrt(-log(tol));
  // Real-space cutoff: up to 15 A, and at most a third of the shortest box side so that the cell
  // path (3 or more cells per axis) applies; not below 9 A (small boxes use the image loop).
  // The k-space work falls as rc^-3 and the real-space work rises as rc^3; with the queued
  // real-space kernel the balance for condensed-phase densities lies near 15 A.
  const double lmin = std::min(box_A[0], std::min(box_A[1], box_A[2]));
  const double rc = std::min(15.0, std::max(9.0, lmin / 3.0 * (1.0 - 1e-6))) / kBohrA;
  g.rc_b = rc;
  g.eta = (x + 0.3) / rc;
  const double kmax = 2.0 * g.eta * x;
  g.vol = 1.0;
  for (int a = 0; a < 3; ++a) {
    g.box_b[a] = box_A[a] / kBohrA;
    g.vol *= g.box_b[a];
    g.nmax[a] = (int)floor(kmax * g.box_b[a] / (2.0 * M_PI));
    g.nimg[a] = (int)floor((rc + 0.5 * g.box_b[a]) / g.box_b[a]);
    g.nc[a] = (int)floor(g.box_b[a] / (rc * (1.0 + 1e-9)));
    g.u[a] = hubbard_u[a];
  }
  g.brute = (g.nc[0] < 3 || g.nc[1] < 3 || g.nc[2] < 3 || g.nimg[0] > 0 || g.nimg[1] > 0 || g.nimg[2] > 0) ? 1 : 0;
  for (int a = 0; a < 3; ++a) if (g.nc[a] < 1) g.nc[a] = 1;
  g.nmax_all = std::max(g.nmax[0], std::max(g.nmax[1], g.nmax[2]));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double si = 1.0 / (sqrt(M_PI) * hubbard_u[i]), sj = 1.0 / (sqrt(M_PI) * hubbard_u[j]);
      g.a[i][j] = 1.0 / sqrt(2.0 * (si * si + sj * sj));
    }
  // k rows (half space)
  std::vector<KRow> rows;
  std::vector<double> wk;
  long long koff = 0;
  const double k2max = kmax * kmax;
  const double tp[3] = {2 * M_PI / g.box_b[0], 2 * M_PI / g.box_b[1], 2 * M_PI / g.box_b[2]};
  m3max_ = 0;
  for (int m1 = 0; m1 <= g.nmax[0]; ++m1)
    for (int m2 = -g.nmax[1]; m2 <= g.nmax[1]; ++m2) {
      if (m1 == 0 && m2 < 0) continue;
      const double k12 = (tp[0] * m1) * (tp[0] * m1) + (tp[1] * m2) * (tp[1] * m2);
      if (k12 > k2max) continue;
      int hi = (int)floor(sqrt((k2max - k12)) / tp[2]);
      hi = std::min(hi, g.nmax[2]);
      int lo = (m1 == 0 && m2 == 0) ? 1 : -hi;
      if (hi < lo) continue;
      KRow r;
      r.m1 = m1; r.m2 = m2; r.m3lo = lo; r.m3hi = hi; r.koff = koff;
      for (int m3 = lo; m3 <= hi; ++m3) {
        const double kz = tp[2] * m3;
        const double k2 = k12 + kz * kz;
        wk.push_back(k2 <= k2max ? 2.0 * (4.0 * M_PI / g.vol) * exp(-k2 / (4.0 * g.eta * g.eta)) / k2 : 0.0);
      }
      koff += hi - lo + 1;
      m3max_ = std::max(m3max_, hi);
      rows.push_back(r);
    }
  nrows_ = (int)rows.size();
  nk_ = koff;
  cudaError_t e;
  if ((e = cudaMalloc(&rows_d, sizeof(KRow) * std::max(1, nrows_)))) return e;
  if ((e = cudaMalloc(&wk_d, sizeof(double) * std::max(1LL, nk_)))) return e;
  cudaMemcpy(rows_d, rows.data(), sizeof(KRow) * nrows_, cudaMemcpyHostToDevice);
  cudaMemcpy(wk_d, wk.data(), sizeof(double) * nk_, cudaMemcpyHostToDevice);
  const size_t csz = fp64 ? sizeof(double2) : sizeof(float2);
  if ((e = cudaMalloc(&tab, csz * 3 * (size_t)N * (g.nmax_all + 1)))) return e;
  nchunk_ = (N + kChunk - 1) / kChunk;
  if ((e = cudaMalloc(&part, sizeof(double) * 2 * 2 * (size_t)nchunk_ * nk_))) return e;
  if ((e = cudaMalloc(&ws, csz * 2 * (size_t)nk_))) return e;
  if ((e = cudaMalloc(&real_buf, sizeof(double) * 3 * N))) return e;
  if ((e = cudaMalloc(&recip_buf, sizeof(double) * 3 * N))) return e;
  if ((e = cudaMalloc(&rpart, sizeof(double) * 3 * (size_t)N * kRowChunks))) return e;
  if ((e = cudaMalloc(&scal, sizeof(double) * 4))) return e;
  const int ncell = g.nc[0] * g.nc[1] * g.nc[2];
  if ((e = cudaMalloc(&cell_of, sizeof(int) * N))) return e;
  if ((e = cudaMalloc(&cell_atoms, sizeof(int) * N))) return e;
  if ((e = cudaMalloc(&cell_count, sizeof(int) * ncell))) return e;
  if ((e = cudaMalloc(&cell_start, sizeof(int) * (ncell + 1)))) return e;
  if ((e = cudaMalloc(&pos_s, sizeof(double4) * N))) return e;
  return cudaSuccess;
}

// The dynamic shared-memory limit of a kernel is a process-wide attribute, while the size a
// launch needs depends on the context's k set: the limit only ever grows (largest request of
// any context so far), so a context never lowers it below what another one launches with.
static std::mutex g_recip_smem_mutex;
static int g_recip_smem[4] = {0, 0, 0, 0};

template <typename T, int MODE>
static void raise_recip_smem(int slot, int bytes) {
  std::lock_guard<std::mutex> lock(g_recip_smem_mutex);
  if (bytes > g_recip_smem[slot]) {
    cudaFuncSetAttribute(recip_atom_kernel<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    g_recip_smem[slot] = bytes;
  }
}

cudaError_t Ewald::prepare(const double* dR, const int* dspecies, cudaStream_t s) {
  const int W = 2 * m3max_ + 1;
  if (fp64_) {
    raise_recip_smem<double, 0>(0, (int)sizeof(double2) * 64 * W);
    raise_recip_smem<double, 1>(1, (int)sizeof(double2) * 64 * W);
  } else {
    raise_recip_smem<float, 0>(2, (int)sizeof(float2) * 128 * W);
    raise_recip_smem<float, 1>(3, (int)sizeof(float2) * 128 * W);
  }
  const int TB = 128, nb = (N_ + TB - 1) / TB;
  if (fp64_) phase_table_kernel<double><<<nb, TB, 0, s>>>(dR, N_, g, reinterpret_cast<double2*>(tab));
  else phase_table_kernel<float><<<nb, TB, 0, s>>>(dR, N_, g, reinterpret_cast<float2*>(tab));
  if (!g.brute) {
    // cell list on the device: counts, scan, stable fill with cell-relative coordinates
    const int ncell = g.nc[0] * g.nc[1] * g.nc[2];
    cudaMemsetAsync(cell_count, 0, sizeof(int) * ncell, s);
    cell_count_kernel<<<nb, TB, 0, s>>>(dR, N_, g, cell_of, cell_count);
    cell_scan_kernel<<<1, 1024, 0, s>>>(cell_count, ncell, cell_start);
    if (fp64_)
      cell_fill_sorted_kernel<double><<<ncell, 256, 0, s>>>(dR, dspecies, N_, g, cell_of, cell_start, cell_atoms,
                                                             reinterpret_cast<double4*>(pos_s));
    else
      cell_fill_sorted_kernel<float><<<ncell, 256, 0, s>>>(dR, dspecies, N_, g, cell_of, cell_start, cell_atoms,
                                                            reinterpret_cast<float4*>(pos_s));
  }
  sb_tag_ = 0;
  dR_ = dR;
  dspecies_ = dspecies;
  return cudaGetLastError();
}

template <typename T>
static void run_sf(Ewald& E, const double* b0, const double* b1, int nv, int vout0, cudaStream_t s) {
  using CT = typename C2<T>::t;
  dim3 grid(E.nrows_, E.nchunk_);
  const size_t shm = sizeof(CT) * Ewald::kChunk * nv + sizeof(T) * 4 * 64 * nv * 2;
  if (nv == 1)
    structure_factor_kernel<T, 1><<<grid, 256, shm, s>>>(E.rows_d, reinterpret_cast<const CT*>(E.tab), b0, b1, E.N_,
                                                        E.g.nmax_all, Ewald::kChunk, E.part, E.nk_);
  else
    structure_factor_kernel<T, 2><<<grid, 256, shm, s>>>(E.rows_d, reinterpret_cast<const CT*>(E.tab), b0, b1, E.N_,
                                                        E.g.nmax_all, Ewald::kChunk, E.part, E.nk_);
  sf_reduce_kernel<T><<<(int)((E.nk_ + 255) / 256), 256, 0, s>>>(E.part, E.nchunk_, nv, E.nk_, E.wk_d,
                                                                 reinterpret_cast<CT*>(E.ws) + (size_t)vout0 * E.nk_);
}

template <typename T, int MODE>
static void run_real(Ewald& E, const double* a, const double* b, cudaStream_t s) {
  if (E.g.brute) {
    real_space_kernel<T, MODE><<<(32 * E.N_ + 127) / 128, 128, 0, s>>>(E.dR_, E.dspecies_, E.N_, E.g, E.cell_start,
                                                                      E.cell_count, E.cell_atoms, E.cell_of, a, b,
                                                                      E.real_buf);
  } else {
    real_cells_kernel<T, MODE><<<(E.N_ + 3) / 4, 128, 0, s>>>(
        reinterpret_cast<const typename Pos4<T>::t*>(E.pos_s), E.cell_atoms, E.cell_start, E.N_, E.g, a, b,
        E.real_buf);
  }
}

cudaError_t Ewald::potential(const double* b, double* V, cudaStream_t s, int tag) {
  const int TB = 128, nb = (N_ + TB - 1) / TB;
  const int W = 2 * m3max_ + 1;
  if (fp64_) {
    run_sf<double>(*this, b, nullptr, 1, 0, s);
    run_real<double, 0>(*this, nullptr, b, s);
    const int tpb = 64;
    recip_atom_kernel<double, 0><<<dim3((N_ + tpb - 1) / tpb, kRowChunks), tpb, sizeof(double2) * tpb * W, s>>>(
        rows_d, nrows_, reinterpret_cast<const double2*>(tab), reinterpret_cast<const double2*>(ws), nk_, N_,
        g.nmax_all, m3max_, g, nullptr, nullptr, rpart);
    chunk_reduce_kernel<<<(N_ + 255) / 256, 256, 0, s>>>(rpart, kRowChunks, N_, recip_buf);
  } else {
    run_sf<float>(*this, b, nullptr, 1, 0, s);
    run_real<float, 0>(*this, nullptr, b, s);
    const int tpb = 128;
    recip_atom_kernel<float, 0><<<dim3((N_ + tpb - 1) / tpb, kRowChunks), tpb, sizeof(float2) * tpb * W, s>>>(
        rows_d, nrows_, reinterpret_cast<const float2*>(tab), reinterpret_cast<const float2*>(ws), nk_, N_,
        g.nmax_all, m3max_, g, nullptr, nullptr, rpart);
    chunk_reduce_kernel<<<(N_ + 255) / 256, 256, 0, s>>>(rpart, kRowChunks, N_, recip_buf);
  }
  sb_tag_ = tag;
  sum_kernel<<<1, 1024, 0, s>>>(b, N_, scal);
  combine_pot_kernel<<<nb, TB, 0, s>>>(real_buf, recip_buf, b, dspecies_, g, scal, V, N_);
  return cudaGetLastError();
}

cudaError_t Ewald::gradient(const double* a, const double* b, double* G, cudaStream_t s, int tag) {
  const int W = 2 * m3max_ + 1;
  // vector 0 = b (S_b), vector 1 = a (S_a); S_b is kept from the potential call with the same
  // nonzero tag (same charges at the same geometry)
  const bool reuse = tag != 0 && tag == sb_tag_;
  if (fp64_) {
    if (reuse) run_sf<double>(*this, a, nullptr, 1, 1, s);
    else run_sf<double>(*this, b, a, 2, 0, s);
    run_real<double, 1>(*this, a, b, s);
    const int tpb = 64;
    recip_atom_kernel<double, 1><<<dim3((N_ + tpb - 1) / tpb, kRowChunks), tpb, sizeof(double2) * tpb * W, s>>>(
        rows_d, nrows_, reinterpret_cast<const double2*>(tab), reinterpret_cast<const double2*>(ws), nk_, N_,
        g.nmax_all, m3max_, g, a, b, rpart);
    chunk_reduce_kernel<<<(3 * N_ + 255) / 256, 256, 0, s>>>(rpart, kRowChunks, 3LL * N_, recip_buf);
  } else {
    if (reuse) run_sf<float>(*this, a, nullptr, 1, 1, s);
    else run_sf<float>(*this, b, a, 2, 0, s);
    run_real<float, 1>(*this, a, b, s);
    const int tpb = 128;
    recip_atom_kernel<float, 1><<<dim3((N_ + tpb - 1) / tpb, kRowChunks), tpb, sizeof(float2) * tpb * W, s>>>(
        rows_d, nrows_, reinterpret_cast<const float2*>(tab), reinterpret_cast<const float2*>(ws), nk_, N_,
        g.nmax_all, m3max_, g, a, b, rpart);
    chunk_reduce_kernel<<<(3 * N_ + 255) / 256, 256, 0, s>>>(rpart, kRowChunks, 3LL * N_, recip_buf);
  }
  combine_grad_kernel<<<(3 * N_ + 255) / 256, 256, 0, s>>>(real_buf, recip_buf, G, N_, 1.0 / kBohrA);
  return cudaGetLastError();
}

}  // namespace sedacs
