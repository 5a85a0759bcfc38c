// Batched dense kernels on the per-subgraph matrices: problem descriptors shared by the
// tensor-core (split bf16 or fp16 planes, tcgen05) and the FP64 (SIMT) paths.
#pragma once
#include "common.cuh"

namespace sedacs {

// One matrix problem of a batched GEMM
//   C = alpha * A * B^T + beta * I + g1 * C1 + g2 * C2      (generic mode)
// (B^T: B is read by rows, so for the symmetric operands of the method B^T = B; C1, C2 are
// masters added in the epilogue, so a product with I + E is formed as C + C E exactly).  Offsets are bytes from
// the arena base.  For the tensor-core path A and B are blocked split planes (bf16, or the
// two-plane fp16 format) and the master output is fp32 row-major; for the FP64 path every
// matrix is fp64 row-major.
struct GemmMat {
  long long a_off, b_off;        // operand 0-th plane (tensor path) or matrix (fp64 path)
  long long a_plane, b_plane;    // bytes between planes
  long long out_off;             // row-major master output (-1: none)
  long long outp_off;            // blocked planes output (-1: none; tensor path only)
  long long outp_plane;
  long long x_off;               // SP2: master of the current iterate
  long long buf_stride;          // SP2 ping/pong distance (bytes) for a, b, x and the outputs
  long long tr_off;              // SP2: trace partial slots (doubles from the slot base)
  long long c_off;               // response mode: master of X dX; generic mode: C1 (-1: none)
  long long c2_off;              // generic mode: C2 (-1: none)
  int n_pad;                     // row stride of every operand (multiple of 128)
  int m_real;                    // valid output rows
  int n_real;                    // valid output columns
  int k_real;                    // valid inner dimension
  int b_from_sp2;                // generic mode: B taken from the SP2 result buffer
  int a_from_sp2;
  int c_from_sp2;                // generic mode: C1 taken from the SP2 result buffer
  int sym_out;                   // result is symmetric: only tiles tn >= tm are run, each
                                 // off-diagonal tile is also written transposed (not in the
                                 // two-plane fp16 SP2 step, which keeps the upper tiles only)
  int x_planes;                  // SP2 mode, three bf16 or two fp16 planes: the epilogue takes X
                                 // from A's planes (the value the MMAs see), no master
  int c_planes;                  // generic mode: C1 is three blocked bf16 planes at c_off
  long long c_plane;             // bytes between the planes of C1
  long long outp2_off;           // generic mode, second output (planes only; -1: none): with it the
                                 // first output takes alpha * AB^T alone and the second
                                 // alpha2 * AB^T + beta * I + g1 * C1 + g2 * C2
};

struct GemmWork {
  int mat, tm, tn, pad;
};

// Per-subgraph state of the mu-branch SP2 recursion.
struct Sp2State {
  double y;          // image of mu under the polynomial so far
  double t;          // last idempotency error Tr(X - X^2)
  double t1, t2;     // the two errors before it
  double tol;        // stop when t < tol
  double floor_guard;// noise-floor stop applies once t_{k-2} < floor_guard
  int active;        // 1 while iterating
  int iters;         // completed steps
  int cur;           // buffer holding the current iterate
  int kmax;
};

// kModeRsp: first-order response step of the SP2 recursion.  With R1 = X dX (c_off) and the
// product P = dX X: dX <- R1 + P (square branch) or 2 dX - R1 - P (other branch); A, B and
// x (= dX master) are taken from buffer `cur`, the output goes to buffer 1 - cur.
enum GemmMode : int { kModeGeneric = 0, kModeSp2 = 1, kModeRsp = 2 };

struct GemmParams {
  const GemmWork* work;
  const GemmMat* mats;
  uint8_t* arena;
  double* tr_slots;
  Sp2State* sp2;
  int* err;
  int mode;
  int nsplit_out;     // tensor path: plane format written (0: none, 1-3 bf16 planes, 4 two fp16 planes;
                      // the fp16-operand kernel writes two fp16 planes unless 3 is asked for)
  double alpha, beta; // epilogue coefficients (FP64 in the FP64 path, rounded to FP32 on the tensor path)
  double g1, g2;
  double alpha2;      // second output (outp2_off) only
  int ops_upper;      // generic mode, fp16 two-plane path: A and B are symmetric and may be stored as
                      // their upper 128x128 tiles only (blocks left of the diagonal read as transposes)
  int store_upper;    // symmetric result written as its upper tiles only (no mirrored tile)
  int no_master;      // planes only: the FP32 master of the result is not written (no reader needs it)
};

// Host launchers (dense.cu)
void launch_gemm_tc(const GemmParams& p, int n_work, int nsplit, cudaStream_t s);
void launch_gemm_f64(const GemmParams& p, int n_work, cudaStream_t s);

}  // namespace sedacs
