// Batched GEMMs over the per-subgraph matrices.
//
//  * tc_gemm_persistent<NSPLIT, F16>: 5th-generation tensor cores, one persistent CTA per SM,
//    ten warps.  A producer lane streams 16 KB operand blocks (already in the swizzled
//    shared-memory image, see blocked_offset) with bulk copies into a 2-3 stage ring guarded
//    by mbarriers, across tile boundaries; an MMA lane issues tcgen05.mma (M=128, N=128,
//    K=16, fp32 in TMEM) over the split products: bf16 hi*hi (+ hi*mid + mid*hi (+ hi*lo +
//    mid*mid + lo*hi)), or with F16 the fp16 hi*hi + hi*lo + lo*hi of the two-plane format;
//    it commits to the ring's "empty" barriers; eight epilogue warps drain TMEM with
//    tcgen05.ld, hand it back to the MMA lane in three parts for the next tile, and run the
//    epilogue (generic alpha*AB^T + beta*I + g1*C1 + g2*C2, or one step of the mu-branch SP2
//    recursion with its trace partials) writing the fp32 master and / or the split planes of
//    the result, overlapped with the next tile's MMAs.
//  * f64_gemm: the same problems and epilogues in FP64 on the CUDA cores (64x64 tiles).
#include "dense.cuh"

namespace sedacs {

namespace {

template <int NSPLIT>
struct TcCfg {
  static constexpr int kStages = (NSPLIT == 3) ? 2 : 3;
  static constexpr int kStageBytes = 2 * NSPLIT * kBlkBytes;
  static constexpr int kNumProd = (NSPLIT == 1) ? 1 : (NSPLIT == 2 ? 3 : 6);
};

// (a-plane, b-plane) of the kept split products: i + j <= NSPLIT - 1.
__device__ __forceinline__ void prod_planes(int idx, int& pa, int& pb) {
  const int tab_a[6] = {0, 0, 1, 0, 1, 2};
  const int tab_b[6] = {0, 1, 0, 2, 1, 0};
  pa = tab_a[idx];
  pb = tab_b[idx];
}

__device__ __forceinline__ void store_planes8(uint8_t* arena, long long base, long long plane, int fmt,
                                              int n_pad, int row, int col, const float* v) {
  write_planes8(arena, base + blocked_offset(row, col, n_pad), plane, fmt, v);
}

// ------------------------------------------------------------------------------------------
// Persistent, warp-specialised split-plane GEMM.  One CTA per SM walks the work list (128x128
// output tiles) with a stride of gridDim.x.  The producer warp (one lane) streams the operand
// blocks of consecutive tiles through the stage ring without pausing at tile boundaries; the
// MMA warp (one lane) issues the MMAs of a tile once the epilogue has drained the previous
// tile's accumulators; eight epilogue warps prefetch their inputs, drain TMEM into registers,
// release it at once, and then run the epilogue math and stores while the next tile's MMAs
// proceed.  Every wait is bounded.
// ------------------------------------------------------------------------------------------
// Epilogue warps: two per TMEM lane quadrant (warp & 3), each owning one half (warp >> 2)
// of the tile's 128 columns; then one producer warp and one MMA warp.
constexpr int kEpiWarps = 8;
constexpr int kProducerWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1;
constexpr int kTcThreads = 32 * (kEpiWarps + 2);

// Per-warp 32x32 FP32 staging chunk, float4 groups XOR-swizzled by row so that row-wise and
// 8-column-wise float4 accesses spread over all banks.
__device__ __forceinline__ int tb_idx(int r, int c) { return r * 32 + ((((c >> 2) ^ (r & 7))) << 2) + (c & 3); }

template <int NSPLIT>
struct TcPCfg {
  static constexpr int kStages = TcCfg<NSPLIT>::kStages;
  static constexpr int kStageBytes = TcCfg<NSPLIT>::kStageBytes;
  static constexpr int kTransBytes = kEpiWarps * 32 * 32 * 4;
  static constexpr int kSmem = kStages * kStageBytes + kTransBytes + 1024 + 256;
};

// F16: operands in the two-plane fp16 format (NSPLIT = 2): fp16 MMAs, the corrections
// accumulator (hi * lo + lo * hi with the scaled lo) weighted by 2^-11 when drained, and the
// iterate and the output planes in the same format.  In the SP2 step the symmetric iterate is
// kept as its upper 128x128 tiles only: an operand block left of the diagonal, (t, kb) with
// kb / 2 < t, is read as the transpose of the stored block rows of tile (kb / 2, t) (two 8 KB
// halves, MN-major descriptors), and the epilogue writes no mirrored tile.
template <int NSPLIT, bool F16>
__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_persistent(const GemmParams p, int n_work) {
  static_assert(!F16 || NSPLIT == 2, "fp16 operands come as two planes");
  using Cfg = TcCfg<NSPLIT>;
  using PCfg = TcPCfg<NSPLIT>;
  if (*reinterpret_cast<volatile int*>(p.err) & kErrTimeout) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* tbuf = reinterpret_cast<float*>(smem + Cfg::kStages * Cfg::kStageBytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Cfg::kStages * Cfg::kStageBytes + PCfg::kTransBytes);
  uint64_t* empty = full + Cfg::kStages;
  uint64_t* accf = empty + Cfg::kStages;
  // acce[j]: the epilogue has drained hi*hi accumulator j (j = 0 together with the corrections
  // accumulator): the next tile's first k-block writes accumulator 0 and the corrections, the
  // second accumulator 1, the third accumulator 2, so TMEM is handed back in three parts
  uint64_t* acce = accf + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 3);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool stepping = (p.mode == kModeSp2 || p.mode == kModeRsp);
  // operands stored as upper tiles: the SP2 step, and generic products of symmetric operands
  const bool upper_only = F16 && (p.mode == kModeSp2 || p.ops_upper);
  constexpr uint32_t kTmemCols = NSPLIT > 1 ? 512 : 128;

  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    for (int j = 0; j < 3; ++j) mbar_init(&acce[j], kEpiWarps);
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

  if (warp == kProducerWarp) {
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
          if (upper_only) {
            // operand rows t, columns kb: stored block, or rows kb of the stored tile (kb / 2, t)
            auto load_sym = [&](uint8_t* dst, const uint8_t* src, long long plane, int t) {
              if ((kb >> 1) < t) {
                const long long o = ((long long)(kb >> 1) * nkb + 2 * t) * kBlkBytes + (kb & 1) * (kBlkBytes / 2);
#pragma unroll
                for (int pl = 0; pl < NSPLIT; ++pl) {
                  bulk_g2s(dst + pl * kBlkBytes, src + pl * plane + o, kBlkBytes / 2, &full[s]);
                  bulk_g2s(dst + pl * kBlkBytes + kBlkBytes / 2, src + pl * plane + o + kBlkBytes, kBlkBytes / 2,
                           &full[s]);
                }
              } else {
                const long long o = ((long long)t * nkb + kb) * kBlkBytes;
#pragma unroll
                for (int pl = 0; pl < NSPLIT; ++pl) bulk_g2s(dst + pl * kBlkBytes, src + pl * plane + o, kBlkBytes, &full[s]);
              }
            };
            load_sym(st, A, m.a_plane, w.tm);
            load_sym(st + NSPLIT * kBlkBytes, B, m.b_plane, w.tn);
          } else {
#pragma unroll
            for (int pl = 0; pl < NSPLIT; ++pl) {
              bulk_g2s(st + pl * kBlkBytes, A + pl * m.a_plane + aoff, kBlkBytes, &full[s]);
              bulk_g2s(st + (NSPLIT + pl) * kBlkBytes, B + pl * m.b_plane + boff, kBlkBytes, &full[s]);
            }
          }
        }
      }
      // the last copies issued into each stage have landed before shared memory is released
      // (already true on the normal path; bounded on the error path)
      for (long long q = g - 1; q >= 0 && q >= g - Cfg::kStages; --q)
        mbar_wait(&full[q % Cfg::kStages], (uint32_t)((q / Cfg::kStages) & 1));
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      constexpr uint32_t idesc = F16 ? idesc_f16_f32(128, 128) : idesc_bf16_f32(128, 128);
      long long g = 0;
      int ti = 0;
      for (int t = blockIdx.x; t < n_work && ok; t += gridDim.x) {
        const GemmWork w = p.work[t];
        if (!tile_live(w)) continue;
        const GemmMat m = p.mats[w.mat];
        const int kb_end = (m.k_real + 63) >> 6;
        const uint32_t prev = (uint32_t)((ti - 1) & 1);
        // accumulator parts of the previous tile that the next k-block overwrites (all three at
        // once with a single accumulator)
        auto wait_part = [&](int j) -> bool { return ti == 0 || mbar_wait(&acce[j], prev); };
        if (!wait_part(0) || (NSPLIT == 1 && (!wait_part(1) || !wait_part(2)))) { ok = false; break; }
        tc_fence_after();
        for (int kb = 0; kb < kb_end; ++kb, ++g) {
          const int s = (int)(g % Cfg::kStages);
          const long long round = g / Cfg::kStages;
          if (NSPLIT > 1 && (kb == 1 || kb == 2)) {
            if (!wait_part(kb)) { ok = false; break; }
            tc_fence_after();
          }
          if (!mbar_wait(&full[s], (uint32_t)(round & 1))) { ok = false; break; }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + s * Cfg::kStageBytes);
          // operands left of the diagonal arrive transposed (MN-major), see the producer
          const bool a_t = upper_only && (kb >> 1) < w.tm, b_t = upper_only && (kb >> 1) < w.tn;
          const uint32_t id = idesc | (a_t ? kIdescTransA : 0u) | (b_t ? kIdescTransB : 0u);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
            for (int pr = 0; pr < Cfg::kNumProd; ++pr) {
              int pa, pb;
              prod_planes(pr, pa, pb);
              const uint32_t sa = st + pa * kBlkBytes, sb = st + (NSPLIT + pb) * kBlkBytes;
              const uint64_t ad = a_t ? smem_desc_sw128_mn(sa + kk * 2048, kBlkBytes / 2) : smem_desc_sw128(sa + kk * 32);
              const uint64_t bd = b_t ? smem_desc_sw128_mn(sb + kk * 2048, kBlkBytes / 2) : smem_desc_sw128(sb + kk * 32);
              const int hsel = kb % 3;
              const uint32_t acc_col = (NSPLIT == 1) ? 0u : (pr == 0 ? 128u * hsel : 384u);
              uint32_t accum;
              if (NSPLIT == 1) accum = (kb | kk) != 0 ? 1u : 0u;
              else if (pr == 0) accum = (kb >= 3 || kk != 0) ? 1u : 0u;
              else accum = (pr == 1 && (kb | kk) == 0) ? 0u : 1u;
              tc_mma_bf16(tmem + acc_col, ad, bd, id, accum);
            }
          }
          tc_commit(&empty[s]);
        }
        // parts this tile did not write are still consumed, so every barrier advances per tile
        if (NSPLIT > 1 && ok) {
          if (kb_end < 2 && !wait_part(1)) ok = false;
          if (ok && kb_end < 3 && !wait_part(2)) ok = false;
        }
        if (!ok) break;
        tc_commit(accf);
        ++ti;
      }
    }
  } else {
    // ---- epilogue warps --------------------------------------------------------------------
    // TMEM lane quadrant qd (tile rows 32 qd ..), column half hf (tile columns 64 hf ..).  The
    // drain maps a thread to a row; everything global uses the coalesced mapping of 4 lanes
    // per row and 8 consecutive columns per lane (8 rows per instruction).
    const int qd = warp & 3, hf = warp >> 2;
    const int rsub = lane >> 2, csub = (lane & 3) * 8;
    float* tb = tbuf + warp * (32 * 32);
    int ti = 0;
    for (int t = blockIdx.x; t < n_work && ok; t += gridDim.x) {
      const GemmWork w = p.work[t];
      if (!tile_live(w)) continue;
      const GemmMat m = p.mats[w.mat];
      const int cur = tile_cur(w, m);
      const int branch_sq = stepping ? (p.sp2[w.mat].y >= 0.5) : 0;
      const long long in_shift = stepping ? cur * m.buf_stride : 0;
      const long long out_shift = stepping ? (1 - cur) * m.buf_stride : 0;
      const int kb_end = (m.k_real + 63) >> 6;
      const bool diag_tile = (w.tm == w.tn);
      const int row0 = w.tm * 128 + qd * 32;          // first tile row of this warp
      const int colh = w.tn * 128 + hf * 64;          // first tile column of this warp
      // first epilogue input (X for the SP2 / response steps, C1 for the generic form), loaded
      // before the accumulators are ready so that its latency hides behind the MMAs
      const float* in1 = nullptr;
      const uint8_t* in1p = nullptr;                  // ... or its blocked planes
      long long in1_plane = 0;
      if ((NSPLIT == 3 || F16) && p.mode == kModeSp2 && m.x_planes) {
        in1p = p.arena + m.a_off + in_shift;
        in1_plane = m.a_plane;
      } else if (NSPLIT == 3 && !stepping && m.c_planes && m.c_off >= 0) {
        in1p = p.arena + m.c_off + (m.c_from_sp2 ? cur * m.buf_stride : 0);
        in1_plane = m.c_plane;
      } else if (stepping) {
        in1 = reinterpret_cast<const float*>(p.arena + m.x_off + in_shift);
      } else if (m.c_off >= 0) {
        in1 = reinterpret_cast<const float*>(p.arena + m.c_off + (m.c_from_sp2 ? cur * m.buf_stride : 0));
      }
      const float* in2 = nullptr;
      if (p.mode == kModeRsp) in2 = reinterpret_cast<const float*>(p.arena + m.c_off);
      else if (!stepping && m.c2_off >= 0) in2 = reinterpret_cast<const float*>(p.arena + m.c2_off);
      float pre[4][8];
      // the first input of one 32-column chunk in the coalesced mapping (zeros when absent)
      auto load_in1 = [&](int col, float (*dst)[8]) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (F16 && in1p) {
            const long long off = blocked_offset(row0 + 8 * i + rsub, col + csub, m.n_pad);
            const uint4 h = __ldg(reinterpret_cast<const uint4*>(in1p + off));
            const uint4 l = __ldg(reinterpret_cast<const uint4*>(in1p + off + in1_plane));
            const __half* hb = reinterpret_cast<const __half*>(&h);
            const __half* lb = reinterpret_cast<const __half*>(&l);
#pragma unroll
            for (int e = 0; e < 8; ++e) dst[i][e] = join_f16x2(hb[e], lb[e]);
          } else if (in1p) {
            const long long off = blocked_offset(row0 + 8 * i + rsub, col + csub, m.n_pad);
            const uint4 h = __ldg(reinterpret_cast<const uint4*>(in1p + off));
            const uint4 md = __ldg(reinterpret_cast<const uint4*>(in1p + off + in1_plane));
            const uint4 l = __ldg(reinterpret_cast<const uint4*>(in1p + off + 2 * in1_plane));
            const __nv_bfloat16* hb = reinterpret_cast<const __nv_bfloat16*>(&h);
            const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&md);
            const __nv_bfloat16* lb = reinterpret_cast<const __nv_bfloat16*>(&l);
#pragma unroll
            for (int e = 0; e < 8; ++e)
              dst[i][e] = (__bfloat162float(hb[e]) + __bfloat162float(mb[e])) + __bfloat162float(lb[e]);
          } else if (in1) {
            const float* src = in1 + (long long)(row0 + 8 * i + rsub) * m.n_pad + col + csub;
            const float4 a0 = __ldg(reinterpret_cast<const float4*>(src));
            const float4 a1 = __ldg(reinterpret_cast<const float4*>(src + 4));
            dst[i][0] = a0.x; dst[i][1] = a0.y; dst[i][2] = a0.z; dst[i][3] = a0.w;
            dst[i][4] = a1.x; dst[i][5] = a1.y; dst[i][6] = a1.z; dst[i][7] = a1.w;
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) dst[i][e] = 0.f;
          }
        }
      };
      // L2 prefetch of both inputs for this warp's rows and columns while the MMAs run
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const long long ro = (long long)(row0 + 8 * i + rsub) * m.n_pad + colh + csub;
        if (in1) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(in1 + ro));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(in1 + ro + 32));
        }
        if (in1p) {
          // this lane's two 16 B granules of the row in each plane
          const long long o0 = blocked_offset(row0 + 8 * i + rsub, colh + csub, m.n_pad);
          const long long o1 = blocked_offset(row0 + 8 * i + rsub, colh + 32 + csub, m.n_pad);
#pragma unroll
          for (int pl = 0; pl < (F16 ? 2 : 3); ++pl) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(in1p + o0 + pl * in1_plane));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(in1p + o1 + pl * in1_plane));
          }
        }
        if (in2) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(in2 + ro));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(in2 + ro + 32));
        }
      }
      if (!mbar_wait(accf, (uint32_t)(ti & 1))) { ok = false; break; }
      tc_fence_after();
      // drain this warp's 64 columns of the accumulators into registers, handing each part of
      // TMEM back as soon as it is read: accumulator 0 with the corrections, then 1, then 2
      float v[2][32];
      const uint32_t t_row = tmem + ((uint32_t)(qd * 32) << 16);
      auto release = [&](int j) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[j])) : "memory");
      };
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const uint32_t col = (uint32_t)(hf * 64 + cc * 32);
        tmem_ld32(t_row + col, v[cc]);
        if (NSPLIT > 1) {
          float v2[32];
          tmem_ld32(t_row + 384 + col, v2);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[cc][j] = F16 ? fmaf(v2[j], kF16LoInv, v[cc][j]) : v[cc][j] + v2[j];
        }
      }
      release(0);
#pragma unroll
      for (int part = 1; part < 3; ++part) {
        if (NSPLIT > 1 && kb_end > part) {
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            float v2[32];
            tmem_ld32(t_row + 128 * part + (uint32_t)(hf * 64 + cc * 32), v2);
#pragma unroll
            for (int j = 0; j < 32; ++j) v[cc][j] += v2[j];
          }
        }
        release(part);
      }
      ++ti;

      float* outm = (m.out_off >= 0 && !p.no_master) ? reinterpret_cast<float*>(p.arena + m.out_off + out_shift)
                                                     : nullptr;
      const bool planes = m.outp_off >= 0 && p.nsplit_out > 0;
      const int fmt = (F16 && p.nsplit_out != 3) ? kPlanesF16x2 : p.nsplit_out;
      const float e_alpha = (float)p.alpha, e_beta = (float)p.beta, e_g1 = (float)p.g1, e_g2 = (float)p.g2;
      const bool mirror = m.sym_out && !diag_tile && !(F16 && p.mode == kModeSp2) && !p.store_upper;
      const bool dual = !stepping && m.outp2_off >= 0;
      const float e_alpha2 = (float)p.alpha2;
      float tr_x = 0.f, tr_x2 = 0.f;
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int ctile = hf * 64 + cc * 32;            // chunk's first column within the tile
        const int col0 = w.tn * 128 + ctile;
        load_in1(col0, pre);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(tb + tb_idx(lane, 4 * q)) =
              make_float4(v[cc][4 * q], v[cc][4 * q + 1], v[cc][4 * q + 2], v[cc][4 * q + 3]);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int rl = 8 * i + rsub;
          const int grow = row0 + rl;
          const int gcol = col0 + csub;
          float acc[8], out[8];
          {
            const float4 a0 = *reinterpret_cast<const float4*>(tb + tb_idx(rl, csub));
            const float4 a1 = *reinterpret_cast<const float4*>(tb + tb_idx(rl, csub + 4));
            acc[0] = a0.x; acc[1] = a0.y; acc[2] = a0.z; acc[3] = a0.w;
            acc[4] = a1.x; acc[5] = a1.y; acc[6] = a1.z; acc[7] = a1.w;
          }
          float sec[8];
          if (in2) {
            const float* src = in2 + (long long)grow * m.n_pad + gcol;
            const float4 a0 = __ldg(reinterpret_cast<const float4*>(src));
            const float4 a1 = __ldg(reinterpret_cast<const float4*>(src + 4));
            sec[0] = a0.x; sec[1] = a0.y; sec[2] = a0.z; sec[3] = a0.w;
            sec[4] = a1.x; sec[5] = a1.y; sec[6] = a1.z; sec[7] = a1.w;
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) sec[e] = 0.f;
          }
          const bool rok = grow < m.m_real;
          float out2[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const bool ok_ij = rok && (gcol + e) < m.n_real;
            float r;
            if (dual) {
              const float r2 = e_alpha2 * acc[e] + (grow == gcol + e ? e_beta : 0.f) + e_g1 * pre[i][e] + e_g2 * sec[e];
              out2[e] = ok_ij ? r2 : 0.f;
              r = e_alpha * acc[e];
            } else if (stepping) {
              const float sum = acc[e] + sec[e];
              r = branch_sq ? sum : 2.f * pre[i][e] - sum;
              if (p.mode == kModeSp2 && diag_tile && ok_ij && (qd * 32 + rl) == (ctile + csub + e)) {
                tr_x += pre[i][e];
                tr_x2 += acc[e];
              }
            } else {
              r = e_alpha * acc[e] + (grow == gcol + e ? e_beta : 0.f) + e_g1 * pre[i][e] + e_g2 * sec[e];
            }
            out[e] = ok_ij ? r : 0.f;
          }
          const long long goff = (long long)grow * m.n_pad + gcol;
          if (outm) {
            float4* dst = reinterpret_cast<float4*>(outm + goff);
            dst[0] = make_float4(out[0], out[1], out[2], out[3]);
            dst[1] = make_float4(out[4], out[5], out[6], out[7]);
          }
          if (planes) store_planes8(p.arena, m.outp_off + out_shift, m.outp_plane, fmt, m.n_pad, grow, gcol, out);
          if (dual) store_planes8(p.arena, m.outp2_off, m.outp_plane, fmt, m.n_pad, grow, gcol, out2);
          if (mirror) {
            *reinterpret_cast<float4*>(tb + tb_idx(rl, csub)) = make_float4(out[0], out[1], out[2], out[3]);
            *reinterpret_cast<float4*>(tb + tb_idx(rl, csub + 4)) = make_float4(out[4], out[5], out[6], out[7]);
          }
        }
        if (mirror) {
          // mirrored tile: output row (col0 + j) takes column j of the chunk
          __syncwarp();
#pragma unroll 1
          for (int i = 0; i < 4; ++i) {
            const int jl = 8 * i + rsub;
            const int trow = col0 + jl;
            const int tcol = row0 + csub;
            float tv[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) tv[e] = tb[tb_idx(csub + e, jl)];
            const long long toff = (long long)trow * m.n_pad + tcol;
            if (outm) {
              float4* dst = reinterpret_cast<float4*>(outm + toff);
              dst[0] = make_float4(tv[0], tv[1], tv[2], tv[3]);
              dst[1] = make_float4(tv[4], tv[5], tv[6], tv[7]);
            }
            if (planes) store_planes8(p.arena, m.outp_off + out_shift, m.outp_plane, fmt, m.n_pad, trow, tcol, tv);
          }
        }
      }
      if (p.mode == kModeSp2 && diag_tile && (qd >> 1) == hf) {
        // the warp holding the diagonal of quadrant qd writes its slot pair (summed in fixed
        // order by the control kernel)
        const float sx = warp_sumf(tr_x), sx2 = warp_sumf(tr_x2);
        if (lane == 0) {
          p.tr_slots[m.tr_off + 8 * w.tm + 2 * qd] = sx;
          p.tr_slots[m.tr_off + 8 * w.tm + 2 * qd + 1] = sx2;
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
        v = p.alpha * acc[i][j] + (row == col ? p.beta : 0.0);
        if (m.c_off >= 0)
          v += p.g1 * reinterpret_cast<const double*>(
                   p.arena + m.c_off + (m.c_from_sp2 ? cur * m.buf_stride : 0))[(long long)row * ld + col];
        if (m.c2_off >= 0) v += p.g2 * reinterpret_cast<const double*>(p.arena + m.c2_off)[(long long)row * ld + col];
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

template <int NSPLIT, bool F16 = false>
static void launch_tc(const GemmParams& p, int n_work, cudaStream_t s) {
  static bool init = false;
  if (!init) {
    cudaFuncSetAttribute(tc_gemm_persistent<NSPLIT, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
  tc_gemm_persistent<NSPLIT, F16><<<grid, kTcThreads, TcPCfg<NSPLIT>::kSmem, s>>>(p, n_work);
}

void launch_gemm_tc(const GemmParams& p, int n_work, int nsplit, cudaStream_t s) {
  if (n_work <= 0) return;
  switch (nsplit) {
    case 1: launch_tc<1>(p, n_work, s); break;
    case 2: launch_tc<2>(p, n_work, s); break;
    case kPlanesF16x2: launch_tc<2, true>(p, n_work, s); break;
    default: launch_tc<3>(p, n_work, s); break;
  }
}

void launch_gemm_f64(const GemmParams& p, int n_work, cudaStream_t s) {
  if (n_work <= 0) return;
  f64_gemm_kernel<<<n_work, 256, 0, s>>>(p);
}

}  // namespace sedacs
