// Batched GEMMs over the per-subgraph matrices.
//
//  * tc_gemm_persistent<NSPLIT>: 5th-generation tensor cores, one persistent CTA per SM,
//    six warps.  A producer lane streams 16 KB operand blocks (already in the swizzled
//    shared-memory image, see blocked_offset) with bulk copies into a 2-3 stage ring guarded
//    by mbarriers, across tile boundaries; an MMA lane issues tcgen05.mma (M=128, N=128,
//    K=16, bf16 in, fp32 in TMEM) over the split products hi*hi (+ hi*mid + mid*hi (+ hi*lo
//    + mid*mid + lo*hi)) and commits to the ring's "empty" barriers; four epilogue warps
//    drain TMEM with tcgen05.ld, hand it back to the MMA lane for the next tile, and run the
//    epilogue (generic alpha*AB^T + beta*I + g1*C1 + g2*C2, or one step of the mu-branch SP2
//    recursion with its trace partials) writing the fp32 master and the split planes of the
//    result, overlapped with the next tile's MMAs.
//  * f64_gemm: the same problems and epilogues in FP64 on the CUDA cores (64x64 tiles).
#include "dense.cuh"

namespace sedacs {

namespace {

template <int NSPLIT>
struct TcCfg {
  static constexpr int kStages = (NSPLIT == 3) ? 2 : 3;
  static constexpr int kStageBytes = 2 * NSPLIT * kBlkBytes;
  static constexpr int kSmem = kStages * kStageBytes + 1024 + 256;
  static constexpr int kNumProd = (NSPLIT == 1) ? 1 : (NSPLIT == 2 ? 3 : 6);
};

// (a-plane, b-plane) of the kept split products: i + j <= NSPLIT - 1.
__device__ __forceinline__ void prod_planes(int idx, int& pa, int& pb) {
  const int tab_a[6] = {0, 0, 1, 0, 1, 2};
  const int tab_b[6] = {0, 1, 0, 2, 1, 0};
  pa = tab_a[idx];
  pb = tab_b[idx];
}

__device__ __forceinline__ void store_planes8(uint8_t* arena, long long base, long long plane, int nsplit,
                                              int n_pad, int row, int col, const float* v) {
  __align__(16) __nv_bfloat16 h[8], m[8], l[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) split3(v[e], h[e], m[e], l[e]);
  const long long off = base + blocked_offset(row, col, n_pad);
  *reinterpret_cast<uint4*>(arena + off) = *reinterpret_cast<const uint4*>(h);
  if (nsplit > 1) *reinterpret_cast<uint4*>(arena + off + plane) = *reinterpret_cast<const uint4*>(m);
  if (nsplit > 2) *reinterpret_cast<uint4*>(arena + off + 2 * plane) = *reinterpret_cast<const uint4*>(l);
}

// ------------------------------------------------------------------------------------------
// Persistent, warp-specialised split-bf16 GEMM.  One CTA per SM walks the work list (128x128
// output tiles) with a stride of gridDim.x.  Warp 4 (one lane) streams the operand blocks of consecutive
// tiles through the stage ring without pausing at tile boundaries; warp 5 (one lane) issues
// the MMAs of a tile once the epilogue has drained the previous tile's accumulators; warps
// 0-3 drain TMEM into registers, release it at once, and then run the epilogue math and stores
// while the next tile's MMAs proceed.  Every wait is bounded.
// ------------------------------------------------------------------------------------------
template <int NSPLIT>
struct TcPCfg {
  static constexpr int kStages = TcCfg<NSPLIT>::kStages;
  static constexpr int kStageBytes = TcCfg<NSPLIT>::kStageBytes;
  static constexpr int kTransBytes = 4 * 32 * 33 * 4;
  static constexpr int kSmem = kStages * kStageBytes + kTransBytes + 1024 + 256;
};

template <int NSPLIT>
__global__ void __launch_bounds__(192, 1) tc_gemm_persistent(const GemmParams p, int n_work) {
  using Cfg = TcCfg<NSPLIT>;
  using PCfg = TcPCfg<NSPLIT>;
  if (*reinterpret_cast<volatile int*>(p.err) & kErrTimeout) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* tbuf = reinterpret_cast<float*>(smem + Cfg::kStages * Cfg::kStageBytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Cfg::kStages * Cfg::kStageBytes + PCfg::kTransBytes);
  uint64_t* empty = full + Cfg::kStages;
  uint64_t* accf = empty + Cfg::kStages;
  uint64_t* acce = accf + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool stepping = (p.mode == kModeSp2 || p.mode == kModeRsp);
  constexpr uint32_t kTmemCols = NSPLIT > 1 ? 512 : 128;

  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, 4);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  // tiles of finished SP2 subgraphs are skipped by every role alike
  auto tile_live = [&](const GemmWork& w) -> bool { return !stepping || p.sp2[w.mat].active; };
  auto tile_cur = [&](const GemmWork& w, const GemmMat& m) -> int {
    return (stepping || m.b_from_sp2 || m.a_from_sp2 || m.c_from_sp2) ? p.sp2[w.mat].cur : 0;
  };

  if (warp == 4) {
    if (lane == 0) {
      long long g = 0;
      for (int t = blockIdx.x; t < n_work && ok; t += gridDim.x) {
        const GemmWork w = p.work[t];
        if (!tile_live(w)) continue;
        const GemmMat m = p.mats[w.mat];
        const int cur = tile_cur(w, m);
        const long long in_shift = stepping ? cur * m.buf_stride : 0;
        const uint8_t* A = p.arena + m.a_off + (stepping ? in_shift : (m.a_from_sp2 ? cur * m.buf_stride : 0));
        const uint8_t* B = p.arena + m.b_off + (stepping ? in_shift : (m.b_from_sp2 ? cur * m.buf_stride : 0));
        const int nkb = m.n_pad >> 6, kb_end = (m.k_real + 63) >> 6;
        for (int kb = 0; kb < kb_end; ++kb, ++g) {
          const int s = (int)(g % Cfg::kStages);
          const long long round = g / Cfg::kStages;
          if (g >= Cfg::kStages && !mbar_wait(&empty[s], (uint32_t)((round - 1) & 1))) { ok = false; break; }
          mbar_arrive_expect_tx(&full[s], Cfg::kStageBytes);
          uint8_t* st = smem + s * Cfg::kStageBytes;
          const long long aoff = ((long long)w.tm * nkb + kb) * kBlkBytes;
          const long long boff = ((long long)w.tn * nkb + kb) * kBlkBytes;
#pragma unroll
          for (int pl = 0; pl < NSPLIT; ++pl) {
            bulk_g2s(st + pl * kBlkBytes, A + pl * m.a_plane + aoff, kBlkBytes, &full[s]);
            bulk_g2s(st + (NSPLIT + pl) * kBlkBytes, B + pl * m.b_plane + boff, kBlkBytes, &full[s]);
          }
        }
      }
      // the last copies issued into each stage have landed before shared memory is released
      // (already true on the normal path; bounded on the error path)
      for (long long q = g - 1; q >= 0 && q >= g - Cfg::kStages; --q)
        mbar_wait(&full[q % Cfg::kStages], (uint32_t)((q / Cfg::kStages) & 1));
    }
  } else if (warp == 5) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(128, 128);
      long long g = 0;
      int ti = 0;
      for (int t = blockIdx.x; t < n_work && ok; t += gridDim.x) {
        const GemmWork w = p.work[t];
        if (!tile_live(w)) continue;
        const GemmMat m = p.mats[w.mat];
        const int kb_end = (m.k_real + 63) >> 6;
        if (ti > 0 && !mbar_wait(acce, (uint32_t)((ti - 1) & 1))) { ok = false; break; }
        tc_fence_after();
        for (int kb = 0; kb < kb_end; ++kb, ++g) {
          const int s = (int)(g % Cfg::kStages);
          const long long round = g / Cfg::kStages;
          if (!mbar_wait(&full[s], (uint32_t)(round & 1))) { ok = false; break; }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + s * Cfg::kStageBytes);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
            for (int pr = 0; pr < Cfg::kNumProd; ++pr) {
              int pa, pb;
              prod_planes(pr, pa, pb);
              const uint64_t ad = smem_desc_sw128(st + pa * kBlkBytes + kk * 32);
              const uint64_t bd = smem_desc_sw128(st + (NSPLIT + pb) * kBlkBytes + kk * 32);
              const int hsel = kb % 3;
              const uint32_t acc_col = (NSPLIT == 1) ? 0u : (pr == 0 ? 128u * hsel : 384u);
              uint32_t accum;
              if (NSPLIT == 1) accum = (kb | kk) != 0 ? 1u : 0u;
              else if (pr == 0) accum = (kb >= 3 || kk != 0) ? 1u : 0u;
              else accum = (pr == 1 && (kb | kk) == 0) ? 0u : 1u;
              tc_mma_bf16(tmem + acc_col, ad, bd, idesc, accum);
            }
          }
          tc_commit(&empty[s]);
        }
        tc_commit(accf);
        ++ti;
      }
    }
  } else {
    // ---- epilogue warps 0-3: thread = output row of the tile ---------------------------------
    int ti = 0;
    float* tb = tbuf + warp * (32 * 33);
    for (int t = blockIdx.x; t < n_work && ok; t += gridDim.x) {
      const GemmWork w = p.work[t];
      if (!tile_live(w)) continue;
      const GemmMat m = p.mats[w.mat];
      const int cur = tile_cur(w, m);
      const int branch_sq = (p.mode == kModeSp2 || p.mode == kModeRsp) ? (p.sp2[w.mat].y >= 0.5) : 0;
      const long long in_shift = stepping ? cur * m.buf_stride : 0;
      const long long out_shift = stepping ? (1 - cur) * m.buf_stride : 0;
      const int kb_end = (m.k_real + 63) >> 6;
      const int row_local = warp * 32 + lane;
      const int row = w.tm * 128 + row_local;
      const bool row_ok = row < m.m_real;
      const bool diag_tile = (w.tm == w.tn);
      {
        const long long roff = ((long long)row * m.n_pad + w.tn * 128) * 4;
        const uint8_t* pre[3] = {nullptr, nullptr, nullptr};
        if (stepping) pre[0] = p.arena + m.x_off + in_shift + roff;
        if (p.mode == kModeRsp) pre[1] = p.arena + m.c_off + roff;
        if (p.mode == kModeGeneric && m.c_off >= 0)
          pre[1] = p.arena + m.c_off + (m.c_from_sp2 ? cur * m.buf_stride : 0) + roff;
        if (p.mode == kModeGeneric && m.c2_off >= 0) pre[2] = p.arena + m.c2_off + roff;
        if (row_ok)
          for (int u = 0; u < 3; ++u)
            if (pre[u])
#pragma unroll
              for (int q = 0; q < 4; ++q) asm volatile("prefetch.global.L2 [%0];" ::"l"(pre[u] + q * 128));
      }
      if (!mbar_wait(accf, (uint32_t)(ti & 1))) { ok = false; break; }
      tc_fence_after();
      // drain every accumulator of this tile into registers, then hand TMEM back
      float v[4][32];
      const uint32_t t_row = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        tmem_ld32(t_row + c * 32, v[c]);
        if (NSPLIT > 1) {
          float v2[32];
          if (kb_end > 1) {
            tmem_ld32(t_row + 128 + c * 32, v2);
#pragma unroll
            for (int j = 0; j < 32; ++j) v[c][j] += v2[j];
          }
          if (kb_end > 2) {
            tmem_ld32(t_row + 256 + c * 32, v2);
#pragma unroll
            for (int j = 0; j < 32; ++j) v[c][j] += v2[j];
          }
          tmem_ld32(t_row + 384 + c * 32, v2);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[c][j] += v2[j];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(acce)) : "memory");
      ++ti;

      float* outm = (m.out_off >= 0) ? reinterpret_cast<float*>(p.arena + m.out_off + out_shift) : nullptr;
      const float* xm = stepping ? reinterpret_cast<const float*>(p.arena + m.x_off + in_shift) : nullptr;
      const float* cm = (p.mode == kModeRsp) ? reinterpret_cast<const float*>(p.arena + m.c_off) : nullptr;
      float tr_x = 0.f, tr_x2 = 0.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float* vv = v[c];
        const int col0 = w.tn * 128 + c * 32;
        if (p.mode == kModeRsp) {
          const float4* sx = reinterpret_cast<const float4*>(xm + (long long)row * m.n_pad + col0);
          const float4* sc = reinterpret_cast<const float4*>(cm + (long long)row * m.n_pad + col0);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 a = sx[q], c4 = sc[q];
            const float xa[4] = {a.x, a.y, a.z, a.w}, ca[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int j = 4 * q + e;
              const bool ok_ij = row_ok && (col0 + j) < m.n_real;
              const float sum = vv[j] + ca[e];
              vv[j] = ok_ij ? (branch_sq ? sum : 2.f * xa[e] - sum) : 0.f;
            }
          }
        } else if (p.mode == kModeSp2) {
          float x[32];
          const float4* src = reinterpret_cast<const float4*>(xm + (long long)row * m.n_pad + col0);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 t4 = src[q];
            x[4 * q] = t4.x; x[4 * q + 1] = t4.y; x[4 * q + 2] = t4.z; x[4 * q + 3] = t4.w;
          }
          if (diag_tile && c == warp && row_ok) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j == lane) { tr_x = x[j]; tr_x2 = vv[j]; }
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const bool ok_ij = row_ok && (col0 + j) < m.n_real;
            const float nv = branch_sq ? vv[j] : 2.f * x[j] - vv[j];
            vv[j] = ok_ij ? nv : 0.f;
          }
        } else {
          float c1[32], c2[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) { c1[j] = 0.f; c2[j] = 0.f; }
          if (m.c_off >= 0) {
            const float4* s1 = reinterpret_cast<const float4*>(
                p.arena + m.c_off + (m.c_from_sp2 ? cur * m.buf_stride : 0) + ((long long)row * m.n_pad + col0) * 4);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const float4 t4 = s1[q];
              c1[4 * q] = t4.x; c1[4 * q + 1] = t4.y; c1[4 * q + 2] = t4.z; c1[4 * q + 3] = t4.w;
            }
          }
          if (m.c2_off >= 0) {
            const float4* s2 =
                reinterpret_cast<const float4*>(p.arena + m.c2_off + ((long long)row * m.n_pad + col0) * 4);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const float4 t4 = s2[q];
              c2[4 * q] = t4.x; c2[4 * q + 1] = t4.y; c2[4 * q + 2] = t4.z; c2[4 * q + 3] = t4.w;
            }
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = col0 + j;
            const bool ok_ij = row_ok && col < m.n_real;
            vv[j] = ok_ij ? (p.alpha * vv[j] + (row == col ? p.beta : 0.f) + p.g1 * c1[j] + p.g2 * c2[j]) : 0.f;
          }
        }
        if (outm) {
          float4* dst = reinterpret_cast<float4*>(outm + (long long)row * m.n_pad + col0);
#pragma unroll
          for (int q = 0; q < 8; ++q) dst[q] = make_float4(vv[4 * q], vv[4 * q + 1], vv[4 * q + 2], vv[4 * q + 3]);
        }
        if (m.outp_off >= 0 && p.nsplit_out > 0) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            store_planes8(p.arena, m.outp_off + out_shift, m.outp_plane, p.nsplit_out, m.n_pad, row, col0 + 8 * q,
                          vv + 8 * q);
        }
        if (m.sym_out && !diag_tile) {
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 32; ++j) tb[lane * 33 + j] = vv[j];
          __syncwarp();
          float tv[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) tv[j] = tb[j * 33 + lane];
          const int trow = col0 + lane;
          const int tcol0 = w.tm * 128 + warp * 32;
          if (outm) {
            float4* dst = reinterpret_cast<float4*>(outm + (long long)trow * m.n_pad + tcol0);
#pragma unroll
            for (int q = 0; q < 8; ++q) dst[q] = make_float4(tv[4 * q], tv[4 * q + 1], tv[4 * q + 2], tv[4 * q + 3]);
          }
          if (m.outp_off >= 0 && p.nsplit_out > 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              store_planes8(p.arena, m.outp_off + out_shift, m.outp_plane, p.nsplit_out, m.n_pad, trow,
                            tcol0 + 8 * q, tv + 8 * q);
          }
        }
      }
      if (p.mode == kModeSp2 && diag_tile) {
        // one slot pair per warp of every diagonal tile (summed in fixed order by the control kernel)
        const float sx = warp_sumf(tr_x), sx2 = warp_sumf(tr_x2);
        if (lane == 0) {
          p.tr_slots[m.tr_off + 8 * w.tm + 2 * warp] = sx;
          p.tr_slots[m.tr_off + 8 * w.tm + 2 * warp + 1] = sx2;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
  if (!ok) atomicOr(p.err, kErrTimeout);
}

// ------------------------------------------------------------------------------------------
// FP64 SIMT batched GEMM, 64x64 tiles, 256 threads (4x4 outputs each), BK = 16.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) f64_gemm_kernel(const GemmParams p) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  __shared__ double red[2][8];
  const GemmWork w = p.work[blockIdx.x];
  const GemmMat m = p.mats[w.mat];
  int cur = 0, branch_sq = 0;
  const bool stepping = (p.mode == kModeSp2 || p.mode == kModeRsp);
  if (stepping) {
    const Sp2State st = p.sp2[w.mat];
    if (!st.active) return;
    cur = st.cur;
    branch_sq = st.y >= 0.5;
  } else if (m.b_from_sp2 || m.a_from_sp2 || m.c_from_sp2) {
    cur = p.sp2[w.mat].cur;
  }
  const long long in_shift = stepping ? cur * m.buf_stride : 0;
  const long long out_shift = stepping ? (1 - cur) * m.buf_stride : 0;
  const double* A = reinterpret_cast<const double*>(
      p.arena + m.a_off + (stepping ? in_shift : (m.a_from_sp2 ? cur * m.buf_stride : 0)));
  const double* B = reinterpret_cast<const double*>(
      p.arena + m.b_off + (stepping ? in_shift : (m.b_from_sp2 ? cur * m.buf_stride : 0)));
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int r0 = w.tm * 64, c0 = w.tn * 64;
  const int ld = m.n_pad;
  double acc[4][4] = {};
  const int k_end = (m.k_real + 15) & ~15;
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  for (int k0 = 0; k0 < k_end; k0 += 16) {
    const double4_32a a4 = *reinterpret_cast<const double4_32a*>(A + (long long)(r0 + lr) * ld + k0 + lk);
    const double4_32a b4 = *reinterpret_cast<const double4_32a*>(B + (long long)(c0 + lr) * ld + k0 + lk);
    As[lk][lr] = a4.x; As[lk + 1][lr] = a4.y; As[lk + 2][lr] = a4.z; As[lk + 3][lr] = a4.w;
    Bs[lk][lr] = b4.x; Bs[lk + 1][lr] = b4.y; Bs[lk + 2][lr] = b4.z; Bs[lk + 3][lr] = b4.w;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { a[i] = As[k][ty * 4 + i]; b[i] = Bs[k][tx * 4 + i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* outm = (m.out_off >= 0) ? reinterpret_cast<double*>(p.arena + m.out_off + out_shift) : nullptr;
  const double* xm = stepping ? reinterpret_cast<const double*>(p.arena + m.x_off + in_shift) : nullptr;
  const double* cm = (p.mode == kModeRsp) ? reinterpret_cast<const double*>(p.arena + m.c_off) : nullptr;
  double tx_ = 0.0, tx2 = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = r0 + ty * 4 + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = c0 + tx * 4 + j;
      const bool ok = row < m.m_real && col < m.n_real;
      double v;
      if (p.mode == kModeSp2) {
        const double x = xm[(long long)row * ld + col];
        if (ok && row == col) { tx_ += x; tx2 += acc[i][j]; }
        v = branch_sq ? acc[i][j] : 2.0 * x - acc[i][j];
      } else if (p.mode == kModeRsp) {
        const double x = xm[(long long)row * ld + col];
        const double sum = acc[i][j] + cm[(long long)row * ld + col];
        v = branch_sq ? sum : 2.0 * x - sum;
      } else {
        v = (double)p.alpha * acc[i][j] + (row == col ? (double)p.beta : 0.0);
        if (m.c_off >= 0)
          v += (double)p.g1 * reinterpret_cast<const double*>(
                   p.arena + m.c_off + (m.c_from_sp2 ? cur * m.buf_stride : 0))[(long long)row * ld + col];
        if (m.c2_off >= 0) v += (double)p.g2 * reinterpret_cast<const double*>(p.arena + m.c2_off)[(long long)row * ld + col];
      }
      if (outm) {
        outm[(long long)row * ld + col] = ok ? v : 0.0;
        if (m.sym_out && w.tm != w.tn) outm[(long long)col * ld + row] = ok ? v : 0.0;
      }
    }
  }
  if (p.mode == kModeSp2 && w.tm == w.tn) {
    const double a = warp_sum(tx_), b = warp_sum(tx2);
    if ((tid & 31) == 0) { red[0][tid >> 5] = a; red[1][tid >> 5] = b; }
    __syncthreads();
    if (tid == 0) {
      double sa = 0.0, sb = 0.0;
      for (int q = 0; q < 8; ++q) { sa += red[0][q]; sb += red[1][q]; }
      p.tr_slots[m.tr_off + 8 * w.tm] = sa;
      p.tr_slots[m.tr_off + 8 * w.tm + 1] = sb;
      for (int q = 2; q < 8; ++q) p.tr_slots[m.tr_off + 8 * w.tm + q] = 0.0;
    }
  }
}

}  // namespace

static int g_num_sms = 0;

template <int NSPLIT>
static void launch_tc(const GemmParams& p, int n_work, cudaStream_t s) {
  static bool init = false;
  if (!init) {
    cudaFuncSetAttribute(tc_gemm_persistent<NSPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         TcPCfg<NSPLIT>::kSmem);
    init = true;
  }
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  const int grid = n_work < g_num_sms ? n_work : g_num_sms;
  tc_gemm_persistent<NSPLIT><<<grid, 192, TcPCfg<NSPLIT>::kSmem, s>>>(p, n_work);
}

void launch_gemm_tc(const GemmParams& p, int n_work, int nsplit, cudaStream_t s) {
  if (n_work <= 0) return;
  switch (nsplit) {
    case 1: launch_tc<1>(p, n_work, s); break;
    case 2: launch_tc<2>(p, n_work, s); break;
    default: launch_tc<3>(p, n_work, s); break;
  }
}

void launch_gemm_f64(const GemmParams& p, int n_work, cudaStream_t s) {
  if (n_work <= 0) return;
  f64_gemm_kernel<<<n_work, 256, 0, s>>>(p);
}

}  // namespace sedacs
