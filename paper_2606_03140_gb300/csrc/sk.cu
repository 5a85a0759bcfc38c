// Slater-Koster sp blocks of the synthetic SCC tight-binding model on the GPU: the padded
// per-subgraph H[n] = H0 + 1/2 (S V + V S) and S gather, and the collected observables
// (Mulliken populations, band energy, atom-condensed density graph, forces).
//
//   V_X(r) = V0_X exp(-r/decay) sw(r),  sw quintic from r_on to r_off,
//   H[s,s] = V_ss, H[s_i,p_a,j] = l_a V_sp, H[p_a,i,s_j] = -l_a V_sp,
//   H[p_a,p_b] = l_a l_b (V_pps - V_ppp) + delta_ab V_ppp,  l = (R_j - R_i)/|R_j - R_i|,
//   S: the same table with every V0 scaled by overlap_scale, unit on-site diagonal
// (Slater & Koster 1954; SCC-DFTB Hamiltonian and overlap, SI Sec. D).  Blocks of an atom
// pair sum every periodic image within r_off (Gamma point).
//
// Collected quantities (Eq. 3 and Sec. "Dynamic Graph Adaption"): for a core atom A of
// subgraph i and every subgraph atom B, with D_c and W_c the core rows of the subgraph
// density and energy-weighted density matrices:
//   pop_A   = sum D_AB . S_AB                (net Mulliken charge dq_A = pop_A - Z_A)
//   eband_A = sum D_AB . H0_AB
//   g_AB    = sum [D dH0 + 1/2 (V_A + V_B) D dS - W dS]_AB  (gradient w.r.t. d = R_B - R_A),
//             dU/dR_A -= g_AB, dU/dR_B += g_AB         (forces at fixed n, Eq. NEQ)
//   G^D_AB  = max |D_AB|.
#include "sk.cuh"

namespace sedacs {

namespace {

template <typename T>
struct Radial {
  T f[5], df[5];   // ss, sp (s on i), ps (s on j), pp sigma, pp pi
};

template <typename T>
__device__ __forceinline__ void radial(const ModelDev& m, int si, int sj, T r, T scale, Radial<T>& o) {
  const T ron = (T)m.r_on, roff = (T)m.r_off, w = roff - ron;
  T sw = 1, dsw = 0;
  if (r > ron) {
    const T t = (r - ron) / w;
    const T t2 = t * t, t3 = t2 * t;
    sw = 1 - 10 * t3 + 15 * t3 * t - 6 * t3 * t2;
    dsw = (-30 * t2 + 60 * t3 - 30 * t3 * t) / w;
  }
  const T e = exp(-r / (T)m.decay);
  const T g = e * sw, dg = e * (dsw - sw / (T)m.decay);
  const T c[5] = {(T)m.v0[si][sj][0], (T)m.v0[si][sj][1], (T)m.v0[sj][si][1], (T)m.v0[si][sj][2],
                  (T)m.v0[si][sj][3]};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    o.f[k] = scale * c[k] * g;
    o.df[k] = scale * c[k] * dg;
  }
}

// Block B[mu][nu] for atoms (i, j) at displacement d = R_j - R_i (Angstrom).
template <typename T>
__device__ __forceinline__ void sk_block(const ModelDev& m, int si, int sj, const T d[3], T scale, T B[4][4]) {
  const T r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  const T l[3] = {d[0] / r, d[1] / r, d[2] / r};
  Radial<T> q;
  radial<T>(m, si, sj, r, scale, q);
  B[0][0] = q.f[0];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    B[0][1 + a] = l[a] * q.f[1];
    B[1 + a][0] = -l[a] * q.f[2];
#pragma unroll
    for (int b = 0; b < 3; ++b) B[1 + a][1 + b] = l[a] * l[b] * (q.f[3] - q.f[4]) + (a == b ? q.f[4] : (T)0);
  }
}

// Contract dB/dd_c with M: out_c = sum_{mu,nu} M[mu][nu] dB_c[mu][nu], for c = 0..2.
template <typename T>
__device__ __forceinline__ void sk_grad_contract(const ModelDev& m, int si, int sj, const T d[3], T scale,
                                                 const T M[4][4], int ni, int nj, T out[3]) {
  const T r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  const T l[3] = {d[0] / r, d[1] / r, d[2] / r};
  Radial<T> q;
  radial<T>(m, si, sj, r, scale, q);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T dl[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) dl[a] = ((a == c ? (T)1 : (T)0) - l[a] * l[c]) / r;
    const T lc = l[c];
    T acc = M[0][0] * q.df[0] * lc;
    if (nj > 1)
#pragma unroll
      for (int a = 0; a < 3; ++a) acc += M[0][1 + a] * (dl[a] * q.f[1] + l[a] * q.df[1] * lc);
    if (ni > 1)
#pragma unroll
      for (int a = 0; a < 3; ++a) acc -= M[1 + a][0] * (dl[a] * q.f[2] + l[a] * q.df[2] * lc);
    if (ni > 1 && nj > 1)
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          T v = (dl[a] * l[b] + l[a] * dl[b]) * (q.f[3] - q.f[4]) + l[a] * l[b] * (q.df[3] - q.df[4]) * lc;
          if (a == b) v += q.df[4] * lc;
          acc += M[1 + a][1 + b] * v;
        }
    out[c] = acc;
  }
}

__device__ __forceinline__ void min_image(const double* R, int i, int j, const double box[3], double d[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double x = R[3 * j + a] - R[3 * i + a];
    d[a] = x - box[a] * rint(x / box[a]);
  }
}

// H0 and S blocks (image sums) for every entry of the pair CSR.
template <typename T>
__global__ void pair_blocks_kernel(const ModelDev m, const double* R, const int* species, const long long* pptr,
                                   const int* pcol, int N, SkGeom g, T* h0b, T* sb) {
  const int A = blockIdx.x;
  const double roff2 = m.r_off * m.r_off;
  for (long long p = pptr[A] + threadIdx.x; p < pptr[A + 1]; p += blockDim.x) {
    const int B = pcol[p];
    double d0[3];
    min_image(R, A, B, g.box, d0);
    T H[4][4] = {}, S[4][4] = {};
    for (int ix = -g.nimg[0]; ix <= g.nimg[0]; ++ix)
      for (int iy = -g.nimg[1]; iy <= g.nimg[1]; ++iy)
        for (int iz = -g.nimg[2]; iz <= g.nimg[2]; ++iz) {
          const double dd[3] = {d0[0] + ix * g.box[0], d0[1] + iy * g.box[1], d0[2] + iz * g.box[2]};
          const double r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
          if (r2 >= roff2 || r2 == 0.0) continue;
          const T dt[3] = {(T)dd[0], (T)dd[1], (T)dd[2]};
          T bh[4][4], bs[4][4];
          sk_block<T>(m, species[A], species[B], dt, (T)1, bh);
          sk_block<T>(m, species[A], species[B], dt, (T)m.overlap_scale, bs);
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) { H[u][v] += bh[u][v]; S[u][v] += bs[u][v]; }
        }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        h0b[p * 16 + u * 4 + v] = H[u][v];
        sb[p * 16 + u * 4 + v] = S[u][v];
      }
  }
}

__global__ void loc_fill_kernel(const long long* sub_ptr, const int* sub_atoms, int* loc, int N) {
  const int i = blockIdx.x;
  int* L = loc + (long long)i * N;
  for (long long q = sub_ptr[i] + threadIdx.x; q < sub_ptr[i + 1]; q += blockDim.x)
    L[sub_atoms[q]] = (int)(q - sub_ptr[i]);
}

// Orbital offsets of every subgraph atom: warp per subgraph, shuffle prefix sums over chunks
// of 32 atoms.
__global__ void orb_offsets_kernel(const long long* sub_ptr, const int* sub_atoms, const int* species, ModelDev m,
                                   int* orb_off, int* n_orb_sub, const int* n_core, int* n_core_orb, int n_sub) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n_sub) return;
  const long long q0 = sub_ptr[i], q1 = sub_ptr[i + 1];
  const int nc = n_core[i];
  int o = 0;                                   // orbitals before this chunk
  for (long long qb = q0; qb < q1; qb += 32) {
    const long long q = qb + lane;
    const int n = q < q1 ? m.n_orb[species[sub_atoms[q]]] : 0;
    int incl = n;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += v;
    }
    if (q < q1) {
      orb_off[q] = o + incl - n;
      if ((int)(q - q0) == nc) n_core_orb[i] = o + incl - n;
    }
    o += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) {
    if ((int)(q1 - q0) == nc) n_core_orb[i] = o;
    n_orb_sub[i] = o;
  }
}

// Padded h (with the Coulomb shift) and s of every subgraph; one warp per subgraph atom row,
// lanes over the atom's pair list, each lane writing one atom-pair block.
template <typename T>
__global__ void gather_kernel(const ModelDev m, const long long* sub_ptr, const int* sub_atoms, const int* orb_off,
                              const int* species, const long long* pptr, const int* pcol, const T* h0b, const T* sb,
                              const int* loc, int N, const double* V, const long long* hoff, const long long* soff,
                              const int* n_pad, uint8_t* arena, int n_sub, const int* sub_of_row,
                              long long total_rows, int shift_only) {
  const long long q = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= total_rows) return;
  const int i = sub_of_row[q];
  const int A = sub_atoms[q];
  const int ld = n_pad[i];
  T* H = reinterpret_cast<T*>(arena + hoff[i]);
  T* Sm = reinterpret_cast<T*>(arena + soff[i]);
  const int sa = species[A];
  const int na = m.n_orb[sa];
  const int oa = orb_off[q];
  const int* L = loc + (long long)i * N;
  const double va = V[A];
  // on-site block: eps + V_A on the diagonal of h, identity in s
  if (lane < na) {
    const int u = lane;
    const long long idx = (long long)(oa + u) * ld + (oa + u);
    H[idx] = (T)((shift_only ? 0.0 : (u == 0 ? m.eps_s[sa] : m.eps_p[sa])) + va);
    Sm[idx] = (T)1;
  }
  for (long long p = pptr[A] + lane; p < pptr[A + 1]; p += 32) {
    const int B = pcol[p];
    const int b = L[B];
    if (b < 0) continue;
    const long long qb = sub_ptr[i] + b;
    const int ob = orb_off[qb];
    const int nb = m.n_orb[species[B]];
    const T shift = (T)(0.5 * (va + V[B]));
    for (int u = 0; u < na; ++u)
      for (int v = 0; v < nb; ++v) {
        const T s = sb[p * 16 + u * 4 + v];
        const long long idx = (long long)(oa + u) * ld + (ob + v);
        H[idx] = (shift_only ? (T)0 : h0b[p * 16 + u * 4 + v]) + shift * s;
        Sm[idx] = s;
      }
  }
}

// Collected observables, one warp per core atom (lanes split its neighbour list; sums are
// combined by a fixed shuffle tree, the reaction on B by FP64 atomics).
template <typename T>
__global__ void observables_kernel(const ModelDev m, const double* R, const int* species, SkGeom g,
                                   const long long* sub_ptr, const int* sub_atoms, const int* orb_off,
                                   const int* core_list, const int* core_sub, const int* core_local, int n_core_total,
                                   const long long* pptr, const int* pcol, const T* h0b, const T* sb, const int* loc,
                                   int N, const double* V, const float* Dc32, const double* Dc64, const float* Wc32,
                                   const double* Wc64, const long long* dc_off, const long long* wc_off, const int* n_pad,
                                   double* pop, double* eband, double* dU, int with_forces) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n_core_total) return;
  const int A = core_list[t], i = core_sub[t], a = core_local[t];
  const long long qa = sub_ptr[i] + a;
  const int sa = species[A], na = m.n_orb[sa], oa = orb_off[qa];
  const int ld = n_pad[i];
  const long long base = dc_off[i] / (Dc64 ? 8 : 4);   // element offset of the core rows
  const long long wbase = wc_off[i] / (Wc64 ? 8 : 4);
  auto Dv = [&](int r, int c) -> double {
    const long long k = base + (long long)r * ld + c;
    return Dc64 ? Dc64[k] : (double)Dc32[k];
  };
  auto Wv = [&](int r, int c) -> double {
    const long long k = wbase + (long long)r * ld + c;
    return Wc64 ? Wc64[k] : (double)Wc32[k];
  };
  const int* L = loc + (long long)i * N;
  double p_acc = 0.0, e_acc = 0.0;
  double fa[3] = {0.0, 0.0, 0.0};
  if (lane == 0)
    for (int u = 0; u < na; ++u) {      // on-site block
      const double d = Dv(oa + u, oa + u);
      p_acc += d;
      e_acc += d * (u == 0 ? m.eps_s[sa] : m.eps_p[sa]);
    }
  const double va = V[A];
  const double roff2 = m.r_off * m.r_off;
  for (long long p = pptr[A] + lane; p < pptr[A + 1]; p += 32) {
    const int B = pcol[p];
    const int b = L[B];
    if (b < 0) continue;
    const int ob = orb_off[sub_ptr[i] + b];
    const int sbp = species[B], nb = m.n_orb[sbp];
    T Dm[4][4] = {}, Wm[4][4] = {};
    for (int u = 0; u < na; ++u)
      for (int v = 0; v < nb; ++v) {
        const double d = Dv(oa + u, ob + v);
        Dm[u][v] = (T)d;
        if (with_forces) Wm[u][v] = (T)Wv(oa + u, ob + v);
        p_acc += d * (double)sb[p * 16 + u * 4 + v];
        e_acc += d * (double)h0b[p * 16 + u * 4 + v];
      }
    if (!with_forces) continue;
    const T vab = (T)(0.5 * (va + V[B]));
    T Ms[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) Ms[u][v] = vab * Dm[u][v] - Wm[u][v];
    double d0[3];
    min_image(R, A, B, g.box, d0);
    double gab[3] = {0.0, 0.0, 0.0};
    for (int ix = -g.nimg[0]; ix <= g.nimg[0]; ++ix)
      for (int iy = -g.nimg[1]; iy <= g.nimg[1]; ++iy)
        for (int iz = -g.nimg[2]; iz <= g.nimg[2]; ++iz) {
          const double dd[3] = {d0[0] + ix * g.box[0], d0[1] + iy * g.box[1], d0[2] + iz * g.box[2]};
          const double r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
          if (r2 >= roff2 || r2 == 0.0) continue;
          const T dt[3] = {(T)dd[0], (T)dd[1], (T)dd[2]};
          T gh[3], gs[3];
          sk_grad_contract<T>(m, sa, sbp, dt, (T)1, Dm, na, nb, gh);
          sk_grad_contract<T>(m, sa, sbp, dt, (T)m.overlap_scale, Ms, na, nb, gs);
#pragma unroll
          for (int c = 0; c < 3; ++c) gab[c] += (double)gh[c] + (double)gs[c];
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      fa[c] -= gab[c];
      atomicAdd(&dU[3 * B + c], gab[c]);
    }
  }
  p_acc = warp_sum(p_acc);
  e_acc = warp_sum(e_acc);
  if (with_forces)
    for (int c = 0; c < 3; ++c) fa[c] = warp_sum(fa[c]);
  if (lane == 0) {
    pop[A] = p_acc;
    eband[A] = e_acc;
    if (with_forces)
      for (int c = 0; c < 3; ++c) atomicAdd(&dU[3 * A + c], fa[c]);
  }
}

// Atom-condensed density graph rows: for core atom A, G^D_AB = max |D_AB| over all subgraph atoms B.
__global__ void gd_kernel(const ModelDev m, const long long* sub_ptr, const int* sub_atoms, const int* orb_off,
                          const int* species, const int* core_list, const int* core_sub, const int* core_local,
                          const float* Dc32, const double* Dc64, const long long* dc_off, const int* n_pad,
                          const long long* gd_ptr, int* gd_col, double* gd_val) {
  const int t = blockIdx.x;
  const int A = core_list[t], i = core_sub[t];
  const long long qa = sub_ptr[i] + core_local[t];
  const int na = m.n_orb[species[A]], oa = orb_off[qa];
  const int ld = n_pad[i];
  const long long base = dc_off[i] / (Dc64 ? 8 : 4);
  const int nsub = (int)(sub_ptr[i + 1] - sub_ptr[i]);
  for (int b = threadIdx.x; b < nsub; b += blockDim.x) {
    const long long qb = sub_ptr[i] + b;
    const int ob = orb_off[qb], nb = m.n_orb[species[sub_atoms[qb]]];
    double mx = 0.0;
    for (int u = 0; u < na; ++u)
      for (int v = 0; v < nb; ++v) {
        const long long k = base + (long long)(oa + u) * ld + (ob + v);
        const double d = Dc64 ? Dc64[k] : (double)Dc32[k];
        mx = fmax(mx, fabs(d));
      }
    gd_col[gd_ptr[A] + b] = sub_atoms[qb];
    gd_val[gd_ptr[A] + b] = mx;
  }
}

// Repulsion energy per atom (1/2 sum) and its gradient, over the pair CSR (images within r_off).
// Warp per atom A, lanes over its pair-list entries, lane sums combined by a fixed shuffle tree.
// T = double: FP64 throughout.  T = float (the FP32 forms): each image term in FP32 from the
// FP64 minimum-image displacement, the sums over pairs in FP64.
template <typename T>
__global__ void repulsion_kernel(const ModelDev m, const double* R, const int* species, SkGeom g,
                                 const long long* pptr, const int* pcol, int N, double* erep_atom, double* dU) {
  const int A = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (A >= N) return;
  double e = 0.0, ga[3] = {0.0, 0.0, 0.0};
  const int sa = species[A];
  const double inv_box[3] = {1.0 / g.box[0], 1.0 / g.box[1], 1.0 / g.box[2]};
  const T r_off = (T)m.r_off, r_on = (T)m.r_on, inv_decay = (T)(1.0 / m.rep_decay);
  for (long long p = pptr[A] + lane; p < pptr[A + 1]; p += 32) {
    const int B = pcol[p];
    const double amp = m.rep_a[sa][species[B]];
    if (amp == 0.0) continue;
    double d0[3];
    if (sizeof(T) == 8) {
      min_image(R, A, B, g.box, d0);
    } else {
      // FP32 form: the minimum image by multiplication (the displacement is needed to FP32 only)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double x = R[3 * B + c] - R[3 * A + c];
        d0[c] = x - g.box[c] * rint(x * inv_box[c]);
      }
    }
    for (int ix = -g.nimg[0]; ix <= g.nimg[0]; ++ix)
      for (int iy = -g.nimg[1]; iy <= g.nimg[1]; ++iy)
        for (int iz = -g.nimg[2]; iz <= g.nimg[2]; ++iz) {
          const T d[3] = {(T)(d0[0] + ix * g.box[0]), (T)(d0[1] + iy * g.box[1]), (T)(d0[2] + iz * g.box[2])};
          const T r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
          if (r >= r_off || r == (T)0) continue;
          T sw = 1, dsw = 0;
          if (r > r_on) {
            const T w = r_off - r_on, t = (r - r_on) / w;
            sw = 1 - 10 * t * t * t + 15 * t * t * t * t - 6 * t * t * t * t * t;
            dsw = (-30 * t * t + 60 * t * t * t - 30 * t * t * t * t) / w;
          }
          const T ex = exp(-r * inv_decay);
          e += 0.5 * amp * (double)(ex * sw);
          const T de = (T)amp * ex * (dsw - sw * inv_decay);
          for (int c = 0; c < 3; ++c) ga[c] -= (double)(de * d[c] / r);
        }
  }
  e = warp_sum(e);
  for (int c = 0; c < 3; ++c) ga[c] = warp_sum(ga[c]);
  if (lane == 0) {
    erep_atom[A] = e;
    for (int c = 0; c < 3; ++c) dU[3 * A + c] += ga[c];
  }
}

}  // namespace

void launch_pair_blocks(const ModelDev& m, const double* R, const int* species, const long long* pptr, const int* pcol,
                        int N, const SkGeom& g, void* h0b, void* sb, bool f64, cudaStream_t s) {
  if (f64) pair_blocks_kernel<double><<<N, 64, 0, s>>>(m, R, species, pptr, pcol, N, g, (double*)h0b, (double*)sb);
  else pair_blocks_kernel<float><<<N, 64, 0, s>>>(m, R, species, pptr, pcol, N, g, (float*)h0b, (float*)sb);
}

void launch_loc_fill(const long long* sub_ptr, const int* sub_atoms, int* loc, int N, int n_sub, cudaStream_t s) {
  cudaMemsetAsync(loc, 0xFF, sizeof(int) * (size_t)N * n_sub, s);
  loc_fill_kernel<<<n_sub, 128, 0, s>>>(sub_ptr, sub_atoms, loc, N);
}

void launch_orb_offsets(const long long* sub_ptr, const int* sub_atoms, const int* species, const ModelDev& m,
                        int* orb_off, int* n_orb_sub, const int* n_core, int* n_core_orb, int n_sub, cudaStream_t s) {
  orb_offsets_kernel<<<(n_sub + 3) / 4, 128, 0, s>>>(sub_ptr, sub_atoms, species, m, orb_off, n_orb_sub, n_core,
                                                     n_core_orb, n_sub);
}

void launch_gather(const ModelDev& m, const long long* sub_ptr, const int* sub_atoms, const int* orb_off,
                   const int* species, const long long* pptr, const int* pcol, const void* h0b, const void* sb,
                   const int* loc, int N, const double* V, const long long* hoff, const long long* soff,
                   const int* n_pad, uint8_t* arena, int n_sub, const int* sub_of_row, long long total_rows,
                   int shift_only, bool f64, cudaStream_t s) {
  const int TB = 128;
  const int nb = (int)((32 * total_rows + TB - 1) / TB);   // warp per subgraph atom row
  if (f64)
    gather_kernel<double><<<nb, TB, 0, s>>>(m, sub_ptr, sub_atoms, orb_off, species, pptr, pcol, (const double*)h0b,
                                            (const double*)sb, loc, N, V, hoff, soff, n_pad, arena, n_sub, sub_of_row,
                                            total_rows, shift_only);
  else
    gather_kernel<float><<<nb, TB, 0, s>>>(m, sub_ptr, sub_atoms, orb_off, species, pptr, pcol, (const float*)h0b,
                                           (const float*)sb, loc, N, V, hoff, soff, n_pad, arena, n_sub, sub_of_row,
                                           total_rows, shift_only);
}

void launch_observables(const ModelDev& m, const double* R, const int* species, const SkGeom& g,
                        const long long* sub_ptr, const int* sub_atoms, const int* orb_off, const int* core_list,
                        const int* core_sub, const int* core_local, int n_core_total, const long long* pptr,
                        const int* pcol, const void* h0b, const void* sb, const int* loc, int N, const double* V,
                        const void* Dc, const void* Wc, const long long* dc_off, const long long* wc_off,
                        const int* n_pad, double* pop, double* eband, double* dU, int with_forces, bool f64,
                        cudaStream_t s) {
  const int TB = 128, nb = (int)((32LL * n_core_total + TB - 1) / TB);
  if (f64)
    observables_kernel<double><<<nb, TB, 0, s>>>(m, R, species, g, sub_ptr, sub_atoms, orb_off, core_list, core_sub,
                                                 core_local, n_core_total, pptr, pcol, (const double*)h0b,
                                                 (const double*)sb, loc, N, V, nullptr, (const double*)Dc, nullptr,
                                                 (const double*)Wc, dc_off, wc_off, n_pad, pop, eband, dU, with_forces);
  else
    observables_kernel<float><<<nb, TB, 0, s>>>(m, R, species, g, sub_ptr, sub_atoms, orb_off, core_list, core_sub,
                                                core_local, n_core_total, pptr, pcol, (const float*)h0b,
                                                (const float*)sb, loc, N, V, (const float*)Dc, nullptr,
                                                (const float*)Wc, nullptr, dc_off, wc_off, n_pad, pop, eband, dU, with_forces);
}

void launch_gd(const ModelDev& m, const long long* sub_ptr, const int* sub_atoms, const int* orb_off,
               const int* species, const int* core_list, const int* core_sub, const int* core_local, int n_core_total,
               const void* Dc, bool f64, const long long* dc_off, const int* n_pad, const long long* gd_ptr, int* gd_col,
               double* gd_val, cudaStream_t s) {
  if (n_core_total <= 0) return;
  gd_kernel<<<n_core_total, 128, 0, s>>>(m, sub_ptr, sub_atoms, orb_off, species, core_list, core_sub, core_local,
                                         f64 ? nullptr : (const float*)Dc, f64 ? (const double*)Dc : nullptr, dc_off,
                                         n_pad, gd_ptr, gd_col, gd_val);
}

void launch_repulsion(const ModelDev& m, const double* R, const int* species, const SkGeom& g, const long long* pptr,
                      const int* pcol, int N, double* erep_atom, double* dU, bool f64, cudaStream_t s) {
  if (f64) repulsion_kernel<double><<<(N + 3) / 4, 128, 0, s>>>(m, R, species, g, pptr, pcol, N, erep_atom, dU);
  else repulsion_kernel<float><<<(N + 3) / 4, 128, 0, s>>>(m, R, species, g, pptr, pcol, N, erep_atom, dU);
}

}  // namespace sedacs
