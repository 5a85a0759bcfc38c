// Elementwise and reduction kernels around the batched GEMMs: split-plane conversion,
// Newton-Schulz start, Gershgorin bounds, the SP2 start matrix and the SP2 step control.
#include "dense_ops.cuh"

namespace sedacs {

namespace {

template <typename T>
__global__ void split_planes_kernel(const SubView* views, uint8_t* arena, int nsplit) {
  const SubView v = views[blockIdx.y];
  const int row = blockIdx.x;
  if (row >= v.rows_pad) return;
  const T* src = reinterpret_cast<const T*>(arena + v.master) + (long long)row * v.n_pad;
  for (int c8 = threadIdx.x * 8; c8 < v.n_pad; c8 += blockDim.x * 8) {
    float x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = (float)src[c8 + e];
    write_planes8(arena, v.planes + blocked_offset(row, c8, v.n_pad), v.plane_stride, nsplit, x);
  }
}

// Affine maps of a master onto one or two outputs, each written as master and / or split
// planes, on the valid block (zero elsewhere): y = a x + b I.  kind 0: (a, b) given; kind 1:
// SP2 start X0 = (emax I - h~) / (emax - emin); kind 2: its first-order change
// dX0 = -dh~ / (emax - emin), with the spectral bounds of each subgraph.  One warp per row,
// 8 consecutive columns per lane (one 16-byte granule of each plane).
struct AffineOut {
  const SubView* views;   // nullptr: no such output
  double a, b;
  int master;             // write the row-major master
  int nsplit;             // plane format to write (0: none)
};

template <typename T>
__global__ void affine_planes_kernel(const SubView* in_v, AffineOut o1, AffineOut o2, int kind, const double* bounds,
                                     uint8_t* arena) {
  const SubView vi = in_v[blockIdx.y];
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= vi.rows_pad) return;
  double a1 = o1.a, b1 = o1.b;
  if (kind != 0) {
    const double emin = bounds[2 * blockIdx.y], emax = bounds[2 * blockIdx.y + 1];
    const double inv = 1.0 / (emax - emin);
    a1 = -inv;
    b1 = kind == 1 ? emax * inv : 0.0;
  }
  const T* src = reinterpret_cast<const T*>(arena + vi.master) + (long long)row * vi.n_pad;
  for (int c8 = lane * 8; c8 < vi.n_pad; c8 += 256) {
    // arithmetic in T (FP32 for the mixed forms: the outputs are FP32 anyway)
    T x[8];
    if (sizeof(T) == 4) {
      const float4 q0 = *reinterpret_cast<const float4*>(src + c8), q1 = *reinterpret_cast<const float4*>(src + c8 + 4);
      x[0] = q0.x; x[1] = q0.y; x[2] = q0.z; x[3] = q0.w; x[4] = q1.x; x[5] = q1.y; x[6] = q1.z; x[7] = q1.w;
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) x[e] = src[c8 + e];
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const AffineOut& o = k == 0 ? o1 : o2;
      if (!o.views) continue;
      const SubView vo = o.views[blockIdx.y];
      const T a = (T)(k == 0 ? a1 : o.a), b = (T)(k == 0 ? b1 : o.b);
      float yf[8];
      T y[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int c = c8 + e;
        const bool ok = row < vi.n_real && c < vi.n_real;
        y[e] = ok ? a * x[e] + (row == c ? b : (T)0) : (T)0;
        yf[e] = (float)y[e];
      }
      if (o.master) {
        T* dst = reinterpret_cast<T*>(arena + vo.master) + (long long)row * vo.n_pad + c8;
        if (sizeof(T) == 4) {
          reinterpret_cast<float4*>(dst)[0] = make_float4(yf[0], yf[1], yf[2], yf[3]);
          reinterpret_cast<float4*>(dst)[1] = make_float4(yf[4], yf[5], yf[6], yf[7]);
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) dst[e] = y[e];
        }
      }
      if (o.nsplit > 0) write_planes8(arena, vo.planes + blocked_offset(row, c8, vo.n_pad), vo.plane_stride, o.nsplit, yf);
    }
  }
}

// Two cubic combinations of E, E^2, E^3 (masters): y_k = a_k E + b_k E^2 + c_k E^3 on the valid
// block, zero elsewhere, each written as master and / or planes.  One warp per row, 8 columns
// per lane.
struct PolyOut {
  const SubView* views;
  double a, b, c;
  int master;
  int nsplit;
};

template <typename T>
__global__ void poly3_kernel(const SubView* e1, const SubView* e2, const SubView* e3, PolyOut o1, PolyOut o2,
                             uint8_t* arena) {
  const SubView v1 = e1[blockIdx.y], v2 = e2[blockIdx.y], v3 = e3[blockIdx.y];
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= v1.rows_pad) return;
  const T* p1 = reinterpret_cast<const T*>(arena + v1.master) + (long long)row * v1.n_pad;
  const T* p2 = reinterpret_cast<const T*>(arena + v2.master) + (long long)row * v2.n_pad;
  const T* p3 = reinterpret_cast<const T*>(arena + v3.master) + (long long)row * v3.n_pad;
  for (int c8 = lane * 8; c8 < v1.n_pad; c8 += 256) {
    T x1[8], x2[8], x3[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      x1[e] = p1[c8 + e];
      x2[e] = p2[c8 + e];
      x3[e] = p3[c8 + e];
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const PolyOut& o = k == 0 ? o1 : o2;
      const SubView vo = o.views[blockIdx.y];
      T y[8];
      float yf[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const bool ok = row < v1.n_real && (c8 + e) < v1.n_real;
        y[e] = ok ? (T)o.a * x1[e] + (T)o.b * x2[e] + (T)o.c * x3[e] : (T)0;
        yf[e] = (float)y[e];
      }
      if (o.master) {
        T* dst = reinterpret_cast<T*>(arena + vo.master) + (long long)row * vo.n_pad + c8;
#pragma unroll
        for (int e = 0; e < 8; ++e) dst[e] = y[e];
      }
      if (o.nsplit > 0) write_planes8(arena, vo.planes + blocked_offset(row, c8, vo.n_pad), vo.plane_stride, o.nsplit, yf);
    }
  }
}

// Gershgorin: per row (one warp), d - r and d + r of the valid block.  FP64 form: every
// magnitude is added in FP64.  FP32 form: each lane sums its n / 32 magnitudes in FP32 and the
// lanes combine in FP64, so that the row costs two FP64 conversions per lane (the FP64 pipe is
// narrow); the radius is then widened by k 2^-23 of itself, more than the relative rounding
// error (k - 1) 2^-24 of a lane's FP32 sum of k = ceil(n / 32) positive terms, so that the disc
// still contains the exact one.
template <typename T>
__global__ void gersh_rows_kernel(const SubView* views, const uint8_t* arena, double* lo, double* hi,
                                  const long long* row_base) {
  const SubView v = views[blockIdx.y];
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= v.n_real) return;
  const T* src = reinterpret_cast<const T*>(arena + v.master) + (long long)row * v.n_pad;
  T s_t = 0, d_t = 0;
  // four consecutive columns per lane and step (rows are 16-byte aligned, padding is zero);
  // unrolled so that a lane's loads of one row are in flight together
#pragma unroll 4
  for (int c4 = lane * 4; c4 < v.n_real; c4 += 128) {
    T x[4];
    if (sizeof(T) == 4) {
      const float4 q = *reinterpret_cast<const float4*>(src + c4);
      x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) x[e] = src[c4 + e];
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int c = c4 + e;
      const T a = c < v.n_real ? x[e] : (T)0;
      if (c == row) d_t = a;
      else s_t += fabs(a);
    }
  }
  double s = warp_sum((double)s_t);
  const double d = warp_sum((double)d_t);
  if (sizeof(T) == 4) s *= 1.0 + (double)((v.n_real + 31) / 32) * 0x1p-23;
  if (lane == 0) {
    lo[row_base[blockIdx.y] + row] = d - s;
    hi[row_base[blockIdx.y] + row] = d + s;
  }
}

__global__ void gersh_reduce_kernel(const SubView* views, const double* lo, const double* hi,
                                    const long long* row_base, double* bounds) {
  const SubView v = views[blockIdx.x];
  double mn = 1e300, mx = -1e300;
  for (int r = threadIdx.x; r < v.n_real; r += blockDim.x) {
    mn = fmin(mn, lo[row_base[blockIdx.x] + r]);
    mx = fmax(mx, hi[row_base[blockIdx.x] + r]);
  }
  __shared__ double smn[256], smx[256];
  smn[threadIdx.x] = mn;
  smx[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      smn[threadIdx.x] = fmin(smn[threadIdx.x], smn[threadIdx.x + o]);
      smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { bounds[2 * blockIdx.x] = smn[0]; bounds[2 * blockIdx.x + 1] = smx[0]; }
}

// X0 = (emax I - h~) / (emax - emin) on the valid block (h~ is stored exactly symmetric:
// its GEMM writes each off-diagonal tile and its transpose from the same values).
__global__ void sp2_replay_init_kernel(Sp2State* st, const double* bounds, const int* n_real, const int* steps,
                                       double mu, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double emin = bounds[2 * i], emax = bounds[2 * i + 1];
  Sp2State s;
  s.y = (emax - mu) / (emax - emin);
  s.t = s.t1 = s.t2 = 0.0;
  s.tol = -1.0;
  s.floor_guard = -1.0;
  s.iters = 0;
  s.cur = 0;
  s.kmax = steps[i];
  s.active = (n_real[i] > 0 && steps[i] > 0) ? 1 : 0;
  st[i] = s;
}

__global__ void sp2_init_kernel(Sp2State* st, const double* bounds, const int* n_real, double mu, double tol,
                                int kmax, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double emin = bounds[2 * i], emax = bounds[2 * i + 1];
  Sp2State s;
  s.y = (emax - mu) / (emax - emin);
  s.t = s.t1 = s.t2 = 0.0;
  s.tol = tol * (double)n_real[i];
  s.floor_guard = 1e-4 * (double)n_real[i];
  s.active = n_real[i] > 0 ? 1 : 0;
  s.iters = 0;
  s.cur = 0;
  s.kmax = kmax;
  st[i] = s;
}

// One step of the recursion control: t_k = Tr(X) - Tr(X^2) from the diagonal-tile slots,
// branch of the image y, stop after the first step with t_k < tol (or kmax steps).
__device__ int sp2_advance_one(Sp2State* st, const double* slots, const long long* tr_off, const int* n_diag,
                               int i) {
  Sp2State s = st[i];
  if (!s.active) return 0;
  double a = 0.0, b = 0.0;
  for (int q = 0; q < 4 * n_diag[i]; ++q) {     // fixed order: tiles, then warps
    a += slots[tr_off[i] + 2 * q];
    b += slots[tr_off[i] + 2 * q + 1];
  }
  s.t2 = s.t1;
  s.t1 = s.t;
  s.t = a - b;
  s.y = (s.y >= 0.5) ? s.y * s.y : 2.0 * s.y - s.y * s.y;
  s.cur ^= 1;
  s.iters += 1;
  // stop on the tolerance, or once the error no longer falls over two steps in the
  // asymptotic regime (rounding noise floor of the arithmetic in use)
  const bool floor_hit = s.iters >= 4 && s.t2 < s.floor_guard && s.t >= s.t2;
  if (s.t < s.tol || floor_hit || s.iters >= s.kmax) s.active = 0;
  st[i] = s;
  return s.active;
}

// One block; *n_active receives the number of subgraphs still active (it may point to mapped
// host memory, which the host reads once the stream has passed this launch).
__global__ void sp2_advance_kernel(Sp2State* st, const double* slots, const long long* tr_off,
                                   const int* n_diag, int* n_active, int n) {
  __shared__ int count;
  if (threadIdx.x == 0) count = 0;
  __syncthreads();
  int mine = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mine += sp2_advance_one(st, slots, tr_off, n_diag, i);
  if (mine) atomicAdd(&count, mine);
  __syncthreads();
  if (threadIdx.x == 0) *reinterpret_cast<volatile int*>(n_active) = count;
}

// fp16 two-plane SP2 iterates (format kPlanesF16x2) of copy `cur` of each subgraph rewritten as
// three bf16 planes (hi + mid + lo of the fp32 value hi + 2^-11 lo, which is exact in fp32) for
// the products that take them next.  The recursion keeps only the upper 128x128 tiles of the
// symmetric iterate, so pass 0 fills each 128x64 block left of the diagonal ((cb / 2) < rb) from
// the transpose of rows 64 (cb & 1) .. of the stored tile (cb / 2, rb), through shared memory;
// pass 1 then converts the stored blocks in place.  One CTA per block.
__global__ void f16x2_to_bf16x3_kernel(const SubView* views, const Sp2State* st, long long copy_stride,
                                       uint8_t* arena, int pass) {
  __shared__ float tr[64][129];
  const SubView v = views[blockIdx.y];
  if (v.planes < 0) return;
  const int nkb = v.n_pad >> 6, nrb = v.rows_pad >> 7;
  const int rb = blockIdx.x / nkb, cb = blockIdx.x % nkb;
  if (rb >= nrb) return;
  const bool lower = (cb >> 1) < rb;
  if (lower != (pass == 0)) return;
  const long long ps = v.plane_stride;
  const long long base = v.planes + (long long)st[blockIdx.y].cur * copy_stride;
  const long long dst = base + ((long long)rb * nkb + cb) * kBlkBytes;
  auto load8 = [&](long long off, float* x) {
    const uint4 hq = *reinterpret_cast<const uint4*>(arena + off);
    const uint4 lq = *reinterpret_cast<const uint4*>(arena + off + ps);
    const __half* h = reinterpret_cast<const __half*>(&hq);
    const __half* l = reinterpret_cast<const __half*>(&lq);
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = join_f16x2(h[e], l[e]);
  };
  if (!lower) {
    for (int g = threadIdx.x; g < kBlkBytes / 16; g += blockDim.x) {   // elementwise: any granule order
      float x[8];
      load8(dst + (long long)g * 16, x);
      write_planes8(arena, dst + (long long)g * 16, ps, 3, x);
    }
    return;
  }
  // source: 64 rows x 128 columns, blocks (cb / 2, 2 rb) and (cb / 2, 2 rb + 1), rows 64 (cb & 1) ..
  const long long src = base + ((long long)(cb >> 1) * nkb + 2 * rb) * kBlkBytes + (cb & 1) * (kBlkBytes / 2);
  for (int g = threadIdx.x; g < 1024; g += blockDim.x) {
    const int sr = g >> 4, half = (g >> 3) & 1, j = g & 7;
    float x[8];
    load8(src + (long long)half * kBlkBytes + sr * 128 + ((j ^ (sr & 7)) << 4), x);
#pragma unroll
    for (int e = 0; e < 8; ++e) tr[sr][half * 64 + j * 8 + e] = x[e];
  }
  __syncthreads();
  // destination row r (source column), columns 8 j .. 8 j + 7 (source rows)
  for (int g = threadIdx.x; g < 1024; g += blockDim.x) {
    const int r = g >> 3, j = g & 7;
    float x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = tr[8 * j + e][r];
    write_planes8(arena, dst + r * 128 + ((j ^ (r & 7)) << 4), ps, 3, x);
  }
}

}  // namespace

void launch_f16x2_to_bf16x3(const SubView* views, const Sp2State* st, long long copy_stride, int n_sub, int max_rows,
                            uint8_t* arena, cudaStream_t s) {
  if (n_sub <= 0 || max_rows <= 0) return;
  dim3 g((max_rows / 128) * (max_rows / 64), n_sub);
  for (int pass = 0; pass < 2; ++pass) f16x2_to_bf16x3_kernel<<<g, 256, 0, s>>>(views, st, copy_stride, arena, pass);
}

void launch_split_planes(const SubView* views, int n_sub, int max_rows, uint8_t* arena, int nsplit, bool f64,
                         cudaStream_t s) {
  if (n_sub <= 0 || max_rows <= 0) return;
  dim3 g(max_rows, n_sub);
  if (f64) split_planes_kernel<double><<<g, 64, 0, s>>>(views, arena, nsplit);
  else split_planes_kernel<float><<<g, 64, 0, s>>>(views, arena, nsplit);
}

void launch_affine_planes(const SubView* in, const SubView* out1, double a1, double b1, int master1, int nsplit1,
                          const SubView* out2, double a2, double b2, int master2, int nsplit2, int kind,
                          const double* bounds, int n_sub, int max_rows, uint8_t* arena, bool f64, cudaStream_t s) {
  if (n_sub <= 0 || max_rows <= 0) return;
  dim3 g((max_rows + 7) / 8, n_sub);
  const AffineOut o1{out1, a1, b1, master1, f64 ? 0 : nsplit1};
  const AffineOut o2{out2, a2, b2, master2, f64 ? 0 : nsplit2};
  if (f64) affine_planes_kernel<double><<<g, 256, 0, s>>>(in, o1, o2, kind, bounds, arena);
  else affine_planes_kernel<float><<<g, 256, 0, s>>>(in, o1, o2, kind, bounds, arena);
}

void launch_poly3(const SubView* e1, const SubView* e2, const SubView* e3, const SubView* out1, double a1, double b1,
                  double c1, int master1, int nsplit1, const SubView* out2, double a2, double b2, double c2,
                  int master2, int nsplit2, int n_sub, int max_rows, uint8_t* arena, bool f64, cudaStream_t s) {
  if (n_sub <= 0 || max_rows <= 0) return;
  dim3 g((max_rows + 7) / 8, n_sub);
  const PolyOut o1{out1, a1, b1, c1, master1, f64 ? 0 : nsplit1};
  const PolyOut o2{out2, a2, b2, c2, master2, f64 ? 0 : nsplit2};
  if (f64) poly3_kernel<double><<<g, 256, 0, s>>>(e1, e2, e3, o1, o2, arena);
  else poly3_kernel<float><<<g, 256, 0, s>>>(e1, e2, e3, o1, o2, arena);
}

void launch_gershgorin(const SubView* views, int n_sub, int max_rows, const uint8_t* arena, double* lo, double* hi,
                       const long long* row_base, double* bounds, bool f64, cudaStream_t s) {
  if (n_sub <= 0) return;
  dim3 g((max_rows + 7) / 8, n_sub);
  if (f64) gersh_rows_kernel<double><<<g, 256, 0, s>>>(views, arena, lo, hi, row_base);
  else gersh_rows_kernel<float><<<g, 256, 0, s>>>(views, arena, lo, hi, row_base);
  gersh_reduce_kernel<<<n_sub, 256, 0, s>>>(views, lo, hi, row_base, bounds);
}

void launch_sp2_replay_init(Sp2State* st, const double* bounds, const int* n_real, const int* steps, double mu, int n,
                            cudaStream_t s) {
  if (n <= 0) return;
  sp2_replay_init_kernel<<<(n + 127) / 128, 128, 0, s>>>(st, bounds, n_real, steps, mu, n);
}

__global__ void buffer_index_kernel(Sp2State* st, int cur, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  st[i].cur = cur;
  st[i].active = 0;
}

void launch_buffer_index(Sp2State* st, int cur, int n, cudaStream_t s) {
  if (n <= 0) return;
  buffer_index_kernel<<<(n + 127) / 128, 128, 0, s>>>(st, cur, n);
}

void launch_sp2_init(Sp2State* st, const double* bounds, const int* n_real, double mu, double tol, int kmax, int n,
                     cudaStream_t s) {
  if (n <= 0) return;
  sp2_init_kernel<<<(n + 127) / 128, 128, 0, s>>>(st, bounds, n_real, mu, tol, kmax, n);
}

void launch_sp2_advance(Sp2State* st, const double* slots, const long long* tr_off, const int* n_diag,
                        int* n_active, int n, cudaStream_t s) {
  if (n <= 0) return;
  sp2_advance_kernel<<<1, 1024, 0, s>>>(st, slots, tr_off, n_diag, n_active, n);
}

}  // namespace sedacs
