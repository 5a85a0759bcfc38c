// Learned charge-response preconditioner on the GPU: a message-passing network on the atom
// graph, linear in the residual y, K_NN(y) = -c y + G(y):
//   h0_i = y_i e[s_i];  a_i = sum_j phi_l(r_ij) * h_j;  h_i <- h_i + A_l a_i + B_l h_i  (3 layers)
//   G(y)_i = w . h3_i;  phi_l(r) = sum_b C_l[b] exp(-((r - m_b)/0.7)^2) (cos(pi r/6) + 1)/2  (r < 6 A)
// 64 channels, FP32.  Forward, backward (parameter gradients with fixed-order reductions)
// and Adam are hand-written kernels; training pairs (x = J v, v) come from the Krylov kernel
// (SI Sec. B).  Parameter order: e[3][64], then per layer C[8][64], A[64][64], B[64][64], then w[64].
#include <cmath>
#include <vector>

#include "engine.cuh"

namespace sedacs {

namespace {

constexpr int W = 64, NB = 8, NL = 3;
constexpr int kParams = 3 * W + NL * (NB * W + 2 * W * W) + W;
constexpr int kAtomsPerBlk = 8;
constexpr float kRcut = 6.0f, kSig = 0.7f;

__host__ __device__ inline int off_e() { return 0; }
__host__ __device__ inline int off_C(int l) { return 3 * W + l * (NB * W + 2 * W * W); }
__host__ __device__ inline int off_A(int l) { return off_C(l) + NB * W; }
__host__ __device__ inline int off_B(int l) { return off_A(l) + W * W; }
__host__ __device__ inline int off_w() { return 3 * W + NL * (NB * W + 2 * W * W); }

// per edge (CSR order): r and the 8 radial basis values with the cosine cutoff
__global__ void edge_basis_kernel(const double* R, const long long* row_ptr, const int* col, int N, double bx,
                                  double by, double bz, float* ebas) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= N) return;
  const double box[3] = {bx, by, bz};
  for (long long p = row_ptr[i] + lane; p < row_ptr[i + 1]; p += 32) {
    const int j = col[p];
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      double d = R[3 * j + a] - R[3 * i + a];
      d -= box[a] * rint(d / box[a]);
      d2 += d * d;
    }
    const float r = (float)sqrt(d2);
    const float fc = r < kRcut ? 0.5f * (cosf(3.14159265358979f * r / kRcut) + 1.0f) : 0.0f;
    for (int b = 0; b < NB; ++b) {
      const float m = 0.8f + (6.0f - 0.8f) * b / (NB - 1);
      const float t = (r - m) / kSig;
      ebas[p * NB + b] = expf(-t * t) * fc;
    }
  }
}

__global__ void embed_kernel(const double* y, const int* species, const float* P, float* h0, int N) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)N * W) return;
  const int i = (int)(t / W), c = (int)(t % W);
  h0[t] = (float)y[i] * P[off_e() + species[i] * W + c];
}

// a_i[c] = sum_{p in row i} (sum_b ebas[p][b] C[b][c]) h[col p][c]; warp per atom, 2 channels per lane.
__global__ void aggregate_kernel(const float* h, const float* P, int l, const long long* row_ptr, const int* col,
                                 const float* ebas, int N, float* a) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= N) return;
  const float* C = P + off_C(l);
  float c0[NB], c1[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) { c0[b] = C[b * W + lane]; c1[b] = C[b * W + lane + 32]; }
  float s0 = 0.f, s1 = 0.f;
  for (long long p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
    const int j = col[p];
    float f0 = 0.f, f1 = 0.f;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const float e = ebas[p * NB + b];
      f0 += e * c0[b];
      f1 += e * c1[b];
    }
    s0 += f0 * h[(long long)j * W + lane];
    s1 += f1 * h[(long long)j * W + lane + 32];
  }
  a[(long long)i * W + lane] = s0;
  a[(long long)i * W + lane + 32] = s1;
}

// out_i[c] = base_i[c] + sum_k M1[c][k] u_i[k] + sum_k M2[c][k] v_i[k]  (trans: use M[k][c])
__global__ void mix_kernel(const float* base, const float* u, const float* v, const float* M1, const float* M2,
                           int trans, int N, float* out) {
  __shared__ float su[kAtomsPerBlk][W], sv[kAtomsPerBlk][W];
  const int c = threadIdx.x;   // 64 threads
  const int i0 = blockIdx.x * kAtomsPerBlk;
  for (int q = 0; q < kAtomsPerBlk; ++q) {
    const int i = i0 + q;
    su[q][c] = i < N ? u[(long long)i * W + c] : 0.f;
    sv[q][c] = (i < N && v) ? v[(long long)i * W + c] : 0.f;
  }
  __syncthreads();
  float acc[kAtomsPerBlk];
  for (int q = 0; q < kAtomsPerBlk; ++q) acc[q] = 0.f;
  for (int k = 0; k < W; ++k) {
    const float m1 = trans ? M1[k * W + c] : M1[c * W + k];
    const float m2 = v ? (trans ? M2[k * W + c] : M2[c * W + k]) : 0.f;
#pragma unroll
    for (int q = 0; q < kAtomsPerBlk; ++q) acc[q] += m1 * su[q][k] + m2 * sv[q][k];
  }
  for (int q = 0; q < kAtomsPerBlk; ++q) {
    const int i = i0 + q;
    if (i < N) out[(long long)i * W + c] = (base ? base[(long long)i * W + c] : 0.f) + acc[q];
  }
}

__global__ void output_kernel(const double* y, const float* h3, const float* P, double c_k0, int N, double* u) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= N) return;
  const float* w = P + off_w();
  float s = h3[(long long)i * W + lane] * w[lane] + h3[(long long)i * W + lane + 32] * w[lane + 32];
  s = warp_sumf(s);
  if (lane == 0) u[i] = -c_k0 * y[i] + (double)s;
}

// gh3_i[c] = gu_i w_c
__global__ void out_bwd_kernel(const double* gu, const float* P, int N, float* gh) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)N * W) return;
  gh[t] = (float)gu[t / W] * P[off_w() + (int)(t % W)];
}

// Partial sums over chunks of atoms (fixed order): part[blk][c*W + k] = sum_i x_i[c] z_i[k].
__global__ void outer_partial_kernel(const float* x, const float* z, int N, int chunk, float* part) {
  const int i0 = blockIdx.x * chunk, i1 = min(N, i0 + chunk);
  for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
    const int c = e / W, k = e % W;
    float s = 0.f;
    for (int i = i0; i < i1; ++i) s += x[(long long)i * W + c] * z[(long long)i * W + k];
    part[(long long)blockIdx.x * W * W + e] = s;
  }
}

// part[blk][c] = sum_i g_i gu_i * h_i[c] ... generic: part[blk][c] = sum_i x_i[c] * s_i (s optional -> 1)
__global__ void vec_partial_kernel(const float* x, const double* s, int N, int chunk, float* part) {
  const int i0 = blockIdx.x * chunk, i1 = min(N, i0 + chunk);
  const int c = threadIdx.x;
  float acc = 0.f;
  for (int i = i0; i < i1; ++i) acc += x[(long long)i * W + c] * (s ? (float)s[i] : 1.f);
  part[blockIdx.x * W + c] = acc;
}

// species embedding gradient partials: part[blk][s*W + c] = sum_{i in chunk, s_i = s} gh0_i[c] y_i
__global__ void embed_bwd_partial_kernel(const float* gh, const double* y, const int* species, int N, int chunk,
                                         float* part) {
  const int i0 = blockIdx.x * chunk, i1 = min(N, i0 + chunk);
  const int c = threadIdx.x;
  float acc[3] = {0.f, 0.f, 0.f};
  for (int i = i0; i < i1; ++i) acc[species[i]] += gh[(long long)i * W + c] * (float)y[i];
  for (int s = 0; s < 3; ++s) part[blockIdx.x * 3 * W + s * W + c] = acc[s];
}

// filter gradient partials: part[blk][b*W + c] = sum_{i in chunk} sum_{p in row i} ebas[p][b] ga_i[c] h_j[c]
__global__ void filter_bwd_partial_kernel(const float* ga, const float* h, const long long* row_ptr, const int* col,
                                          const float* ebas, int N, int chunk, float* part) {
  const int i0 = blockIdx.x * chunk, i1 = min(N, i0 + chunk);
  const int c = threadIdx.x;
  float acc[NB];
  for (int b = 0; b < NB; ++b) acc[b] = 0.f;
  for (int i = i0; i < i1; ++i) {
    const float g = ga[(long long)i * W + c];
    for (long long p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
      const float gh = g * h[(long long)col[p] * W + c];
#pragma unroll
      for (int b = 0; b < NB; ++b) acc[b] += ebas[p * NB + b] * gh;
    }
  }
  for (int b = 0; b < NB; ++b) part[(long long)blockIdx.x * NB * W + b * W + c] = acc[b];
}

// grad[off + e] += sum over blocks of part[blk][e] (fixed order)
__global__ void reduce_partials_kernel(const float* part, int nblk, int len, float scale, float* grad, int off) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= len) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += part[(long long)b * len + e];
  grad[off + e] += scale * s;
}

__global__ void add_f_kernel(float* y, const float* x, long long n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) y[t] += x[t];
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  m[t] = b1 * m[t] + (1.f - b1) * g[t];
  v[t] = b2 * v[t] + (1.f - b2) * g[t] * g[t];
  p[t] -= lr * (m[t] / c1) / (sqrtf(v[t] / c2) + eps);
}

__global__ void residual_kernel(const double* u, const double* v, int N, double scale, double* gu, double* acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) gu[i] = scale * (u[i] - v[i]);
  (void)acc;
}

__global__ void f2d_kernel(const float* x, double* y, long long n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) y[t] = (double)x[t];
}
__global__ void d2f_kernel(const double* x, float* y, long long n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) y[t] = (float)x[t];
}

inline int nb(long long n, int tb) { return (int)((n + tb - 1) / tb); }

}  // namespace

int gnn_num_params() { return kParams; }
void dev_dot_into(sedacs_ctx* ctx, const double* a, const double* b, double* out);

// Parameter, moment and activation buffers (allocated once).
cudaError_t gnn_prepare_params(sedacs_ctx* ctx) {
  GnnState& G = ctx->gnn;
  cudaError_t e;
  const int N = ctx->N;
  if (!G.P) {
    if ((e = cudaMalloc(&G.P, sizeof(float) * kParams))) return e;
    if ((e = cudaMalloc(&G.grad, sizeof(float) * kParams))) return e;
    if ((e = cudaMalloc(&G.m, sizeof(float) * kParams))) return e;
    if ((e = cudaMalloc(&G.v, sizeof(float) * kParams))) return e;
    cudaMemset(G.P, 0, sizeof(float) * kParams);
    cudaMemset(G.m, 0, sizeof(float) * kParams);
    cudaMemset(G.v, 0, sizeof(float) * kParams);
    if ((e = cudaMalloc(&G.act, sizeof(float) * (size_t)N * W * (2 * NL + 4)))) return e;
    G.nchunk = (N + 63) / 64;
    if ((e = cudaMalloc(&G.part, sizeof(float) * (size_t)G.nchunk * W * W))) return e;
    if ((e = cudaMalloc(&G.gu, sizeof(double) * N))) return e;
    if ((e = cudaMalloc(&G.u, sizeof(double) * N))) return e;
  }
  return cudaSuccess;
}

// Edge basis of the current graph (and the buffers above).
cudaError_t gnn_prepare(sedacs_ctx* ctx) {
  GnnState& G = ctx->gnn;
  cudaError_t e;
  const int N = ctx->N;
  if ((e = gnn_prepare_params(ctx))) return e;
  if (ctx->nnz * NB > G.ebas_cap) {
    if (G.ebas) cudaFree(G.ebas);
    G.ebas_cap = ctx->nnz * NB + ctx->nnz * NB / 4 + 1024;
    if ((e = cudaMalloc(&G.ebas, sizeof(float) * G.ebas_cap))) return e;
  }
  edge_basis_kernel<<<nb(32LL * N, 128), 128, 0, ctx->stream>>>(ctx->d_R, ctx->d_row_ptr, ctx->d_col, N, ctx->box[0],
                                                                ctx->box[1], ctx->box[2], G.ebas);
  ctx->launches += 1;
  return cudaGetLastError();
}

// activations layout: h[0..NL] then a[0..NL-1], then two gradient buffers
static float* act(sedacs_ctx* ctx, int k) { return ctx->gnn.act + (size_t)k * ctx->N * W; }

void gnn_forward(sedacs_ctx* ctx, const double* y, double* u) {
  const int N = ctx->N;
  cudaStream_t s = ctx->stream;
  GnnState& G = ctx->gnn;
  embed_kernel<<<nb((long long)N * W, 256), 256, 0, s>>>(y, ctx->d_species, G.P, act(ctx, 0), N);
  for (int l = 0; l < NL; ++l) {
    aggregate_kernel<<<nb(32LL * N, 128), 128, 0, s>>>(act(ctx, l), G.P, l, ctx->d_row_ptr, ctx->d_col, G.ebas, N,
                                                      act(ctx, NL + 1 + l));
    mix_kernel<<<nb(N, kAtomsPerBlk), W, 0, s>>>(act(ctx, l), act(ctx, NL + 1 + l), act(ctx, l), G.P + off_A(l),
                                                 G.P + off_B(l), 0, N, act(ctx, l + 1));
  }
  output_kernel<<<nb(32LL * N, 128), 128, 0, s>>>(y, act(ctx, NL), G.P, ctx->prm.c_k0, N, u);
  ctx->launches += 2 + 2 * NL;
}

// grad += d/dP sum_i gu_i K_NN(y)_i  (forward activations must be current)
void gnn_backward(sedacs_ctx* ctx, const double* y, const double* gu) {
  const int N = ctx->N;
  cudaStream_t s = ctx->stream;
  GnnState& G = ctx->gnn;
  float* gh = act(ctx, 2 * NL + 1);
  float* tmp = act(ctx, 2 * NL + 2);
  const int ch = 64;
  out_bwd_kernel<<<nb((long long)N * W, 256), 256, 0, s>>>(gu, G.P, N, gh);
  vec_partial_kernel<<<G.nchunk, W, 0, s>>>(act(ctx, NL), gu, N, ch, G.part);
  reduce_partials_kernel<<<1, W, 0, s>>>(G.part, G.nchunk, W, 1.f, G.grad, off_w());
  for (int l = NL - 1; l >= 0; --l) {
    float* h = act(ctx, l);
    float* a = act(ctx, NL + 1 + l);
    outer_partial_kernel<<<G.nchunk, 256, 0, s>>>(gh, a, N, ch, G.part);
    reduce_partials_kernel<<<nb(W * W, 256), 256, 0, s>>>(G.part, G.nchunk, W * W, 1.f, G.grad, off_A(l));
    outer_partial_kernel<<<G.nchunk, 256, 0, s>>>(gh, h, N, ch, G.part);
    reduce_partials_kernel<<<nb(W * W, 256), 256, 0, s>>>(G.part, G.nchunk, W * W, 1.f, G.grad, off_B(l));
    // ga = A^T gh  (into tmp); gprev = gh + B^T gh (into gh, via a: a is free after use)
    mix_kernel<<<nb(N, kAtomsPerBlk), W, 0, s>>>(nullptr, gh, nullptr, G.P + off_A(l), nullptr, 1, N, tmp);
    filter_bwd_partial_kernel<<<G.nchunk, W, 0, s>>>(tmp, h, ctx->d_row_ptr, ctx->d_col, G.ebas, N, ch, G.part);
    reduce_partials_kernel<<<nb(NB * W, 256), 256, 0, s>>>(G.part, G.nchunk, NB * W, 1.f, G.grad, off_C(l));
    mix_kernel<<<nb(N, kAtomsPerBlk), W, 0, s>>>(gh, gh, nullptr, G.P + off_B(l), nullptr, 1, N, a);
    // transpose of the aggregation: the graph and the filter are symmetric, so it is an aggregation of ga
    aggregate_kernel<<<nb(32LL * N, 128), 128, 0, s>>>(tmp, G.P, l, ctx->d_row_ptr, ctx->d_col, G.ebas, N, gh);
    add_f_kernel<<<nb((long long)N * W, 256), 256, 0, s>>>(gh, a, (long long)N * W);
  }
  embed_bwd_partial_kernel<<<G.nchunk, W, 0, s>>>(gh, y, ctx->d_species, N, ch, G.part);
  reduce_partials_kernel<<<1, 3 * W, 0, s>>>(G.part, G.nchunk, 3 * W, 1.f, G.grad, off_e());
  ctx->launches += 5 + 9 * NL;
}

void gnn_adam(sedacs_ctx* ctx, float lr) {
  GnnState& G = ctx->gnn;
  G.t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  adam_kernel<<<nb(kParams, 256), 256, 0, ctx->stream>>>(G.P, G.grad, G.m, G.v, kParams, lr, b1, b2, 1e-8f,
                                                        1.f - powf(b1, (float)G.t), 1.f - powf(b2, (float)G.t));
  ctx->launches += 1;
}

void gnn_zero_grad(sedacs_ctx* ctx) { cudaMemsetAsync(ctx->gnn.grad, 0, sizeof(float) * kParams, ctx->stream); }

void gnn_set_params_f64(sedacs_ctx* ctx, const double* d_p) {
  d2f_kernel<<<nb(kParams, 256), 256, 0, ctx->stream>>>(d_p, ctx->gnn.P, kParams);
}
void gnn_get_params_f64(sedacs_ctx* ctx, double* d_p, bool grad) {
  f2d_kernel<<<nb(kParams, 256), 256, 0, ctx->stream>>>(grad ? ctx->gnn.grad : ctx->gnn.P, d_p, kParams);
}

// one Adam step on the mean squared error over n pairs (x_k, v_k), each an N-vector in device
// memory; the loss is read back (one sync per pair) only when want_loss
double gnn_train_step(sedacs_ctx* ctx, const double* X, const double* V, int n, float lr, bool want_loss) {
  const int N = ctx->N;
  cudaStream_t s = ctx->stream;
  GnnState& G = ctx->gnn;
  gnn_zero_grad(ctx);
  std::vector<double> losses(n);
  double* lbuf = ctx->d_scal + 12;
  double loss = 0.0;
  for (int k = 0; k < n; ++k) {
    const double* x = X + (size_t)k * N;
    const double* v = V + (size_t)k * N;
    gnn_forward(ctx, x, G.u);
    residual_kernel<<<nb(N, 256), 256, 0, s>>>(G.u, v, N, 2.0 / n, G.gu, nullptr);
    gnn_backward(ctx, x, G.gu);
    if (!want_loss) continue;
    // loss: sum (u - v)^2 / n  = sum gu^2 * n / 4
    dev_dot_into(ctx, G.gu, G.gu, lbuf);
    double l = 0.0;
    cudaMemcpyAsync(&l, lbuf, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    loss += l * n / 4.0;
  }
  gnn_adam(ctx, lr);
  return loss / n;
}

}  // namespace sedacs
