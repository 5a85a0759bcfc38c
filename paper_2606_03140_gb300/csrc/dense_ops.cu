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
    __align__(16) __nv_bfloat16 h[8], m[8], l[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) split3(x[e], h[e], m[e], l[e]);
    const long long off = v.planes + blocked_offset(row, c8, v.n_pad);
    *reinterpret_cast<uint4*>(arena + off) = *reinterpret_cast<const uint4*>(h);
    if (nsplit > 1) *reinterpret_cast<uint4*>(arena + off + v.plane_stride) = *reinterpret_cast<const uint4*>(m);
    if (nsplit > 2) *reinterpret_cast<uint4*>(arena + off + 2 * v.plane_stride) = *reinterpret_cast<const uint4*>(l);
  }
}

// out = a * in + b * I on the valid block, zero elsewhere (in may alias out).
template <typename T>
__global__ void affine_kernel(const SubView* in_v, const SubView* out_v, uint8_t* arena, double a, double b) {
  const SubView vi = in_v[blockIdx.y];
  const SubView vo = out_v[blockIdx.y];
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);     // one warp per row
  if (row >= vo.rows_pad) return;
  const T* src = reinterpret_cast<const T*>(arena + vi.master) + (long long)row * vi.n_pad;
  T* dst = reinterpret_cast<T*>(arena + vo.master) + (long long)row * vo.n_pad;
  for (int c = threadIdx.x & 31; c < vo.n_pad; c += 32) {
    const bool ok = row < vo.n_real && c < vo.n_real;
    dst[c] = ok ? (T)(a * (double)src[c] + (row == c ? b : 0.0)) : (T)0;
  }
}

// Gershgorin: per row (one warp), d - r and d + r of the valid block.
template <typename T>
__global__ void gersh_rows_kernel(const SubView* views, const uint8_t* arena, double* lo, double* hi,
                                  const long long* row_base) {
  const SubView v = views[blockIdx.y];
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= v.n_real) return;
  const T* src = reinterpret_cast<const T*>(arena + v.master) + (long long)row * v.n_pad;
  double s = 0.0, d = 0.0;
  for (int c = lane; c < v.n_real; c += 32) {
    const double x = (double)src[c];
    if (c == row) d = x; else s += fabs(x);
  }
  s = warp_sum(s);
  d = warp_sum(d);
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
template <typename T>
__global__ void sp2_x0_kernel(const SubView* hv, const SubView* xv, uint8_t* arena, const double* bounds) {
  const SubView vh = hv[blockIdx.y];
  const SubView vx = xv[blockIdx.y];
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= vx.rows_pad) return;
  const double emin = bounds[2 * blockIdx.y], emax = bounds[2 * blockIdx.y + 1];
  const double inv = 1.0 / (emax - emin);
  const T* h = reinterpret_cast<const T*>(arena + vh.master) + (long long)row * vh.n_pad;
  T* x = reinterpret_cast<T*>(arena + vx.master) + (long long)row * vx.n_pad;
  for (int c = threadIdx.x & 31; c < vx.n_pad; c += 32) {
    T out = (T)0;
    if (row < vx.n_real && c < vx.n_real) out = (T)(((row == c ? emax : 0.0) - (double)h[c]) * inv);
    x[c] = out;
  }
}

// dX0 = -dh~ / (emax - emin): first-order change of the SP2 start matrix.
template <typename T>
__global__ void sp2_dx0_kernel(const SubView* hv, const SubView* xv, uint8_t* arena, const double* bounds) {
  const SubView vh = hv[blockIdx.y];
  const SubView vx = xv[blockIdx.y];
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= vx.rows_pad) return;
  const double inv = 1.0 / (bounds[2 * blockIdx.y + 1] - bounds[2 * blockIdx.y]);
  const T* h = reinterpret_cast<const T*>(arena + vh.master) + (long long)row * vh.n_pad;
  T* x = reinterpret_cast<T*>(arena + vx.master) + (long long)row * vx.n_pad;
  for (int c = threadIdx.x & 31; c < vx.n_pad; c += 32) {
    T out = (T)0;
    if (row < vx.n_real && c < vx.n_real) out = (T)(-(double)h[c] * inv);
    x[c] = out;
  }
}

// State of a replay of the recorded SP2 branch sequence (fixed step count per subgraph).
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
__global__ void sp2_advance_kernel(Sp2State* st, const double* slots, const long long* tr_off,
                                   const int* n_diag, int* n_active, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Sp2State s = st[i];
  if (!s.active) return;
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
  else atomicAdd(n_active, 1);
  st[i] = s;
}

}  // namespace

void launch_split_planes(const SubView* views, int n_sub, int max_rows, uint8_t* arena, int nsplit, bool f64,
                         cudaStream_t s) {
  if (n_sub <= 0 || max_rows <= 0) return;
  dim3 g(max_rows, n_sub);
  if (f64) split_planes_kernel<double><<<g, 64, 0, s>>>(views, arena, nsplit);
  else split_planes_kernel<float><<<g, 64, 0, s>>>(views, arena, nsplit);
}

void launch_affine(const SubView* in, const SubView* out, int n_sub, int max_rows, uint8_t* arena, double a,
                   double b, bool f64, cudaStream_t s) {
  if (n_sub <= 0 || max_rows <= 0) return;
  dim3 g((max_rows + 7) / 8, n_sub);
  if (f64) affine_kernel<double><<<g, 256, 0, s>>>(in, out, arena, a, b);
  else affine_kernel<float><<<g, 256, 0, s>>>(in, out, arena, a, b);
}

void launch_gershgorin(const SubView* views, int n_sub, int max_rows, const uint8_t* arena, double* lo, double* hi,
                       const long long* row_base, double* bounds, bool f64, cudaStream_t s) {
  if (n_sub <= 0) return;
  dim3 g((max_rows + 7) / 8, n_sub);
  if (f64) gersh_rows_kernel<double><<<g, 256, 0, s>>>(views, arena, lo, hi, row_base);
  else gersh_rows_kernel<float><<<g, 256, 0, s>>>(views, arena, lo, hi, row_base);
  gersh_reduce_kernel<<<n_sub, 256, 0, s>>>(views, lo, hi, row_base, bounds);
}

void launch_sp2_x0(const SubView* hv, const SubView* xv, int n_sub, int max_rows, uint8_t* arena,
                   const double* bounds, bool f64, cudaStream_t s) {
  if (n_sub <= 0) return;
  dim3 g((max_rows + 7) / 8, n_sub);
  if (f64) sp2_x0_kernel<double><<<g, 256, 0, s>>>(hv, xv, arena, bounds);
  else sp2_x0_kernel<float><<<g, 256, 0, s>>>(hv, xv, arena, bounds);
}

void launch_sp2_dx0(const SubView* hv, const SubView* xv, int n_sub, int max_rows, uint8_t* arena,
                    const double* bounds, bool f64, cudaStream_t s) {
  if (n_sub <= 0) return;
  dim3 g((max_rows + 7) / 8, n_sub);
  if (f64) sp2_dx0_kernel<double><<<g, 256, 0, s>>>(hv, xv, arena, bounds);
  else sp2_dx0_kernel<float><<<g, 256, 0, s>>>(hv, xv, arena, bounds);
}

void launch_sp2_replay_init(Sp2State* st, const double* bounds, const int* n_real, const int* steps, double mu, int n,
                            cudaStream_t s) {
  if (n <= 0) return;
  sp2_replay_init_kernel<<<(n + 127) / 128, 128, 0, s>>>(st, bounds, n_real, steps, mu, n);
}

void launch_sp2_init(Sp2State* st, const double* bounds, const int* n_real, double mu, double tol, int kmax, int n,
                     cudaStream_t s) {
  if (n <= 0) return;
  sp2_init_kernel<<<(n + 127) / 128, 128, 0, s>>>(st, bounds, n_real, mu, tol, kmax, n);
}

void launch_sp2_advance(Sp2State* st, const double* slots, const long long* tr_off, const int* n_diag,
                        int* n_active, int n, cudaStream_t s) {
  if (n <= 0) return;
  sp2_advance_kernel<<<(n + 127) / 128, 128, 0, s>>>(st, slots, tr_off, n_diag, n_active, n);
}

}  // namespace sedacs
