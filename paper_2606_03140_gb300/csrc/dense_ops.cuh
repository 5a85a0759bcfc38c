// Elementwise / reduction helpers on the padded per-subgraph matrices.
#pragma once
#include "dense.cuh"

namespace sedacs {

// Placement of one subgraph's matrix in the arena.
struct SubView {
  long long master;        // row-major master (fp32 or fp64), byte offset
  long long planes;        // blocked bf16 planes (byte offset of plane 0; -1 if none)
  long long plane_stride;  // bytes between planes
  int n_pad;               // row stride (columns)
  int rows_pad;            // stored rows (n_pad for square, 128 * ceil(m/128) for core rows)
  int n_real;              // valid rows = valid columns for square matrices
  int pad;
};

// nsplit: plane format (1-3 bf16 planes, or kPlanesF16x2).
void launch_split_planes(const SubView* views, int n_sub, int max_rows, uint8_t* arena, int nsplit, bool f64,
                         cudaStream_t s);
// Rewrite the kPlanesF16x2 planes of copy st[i].cur of every subgraph, stored as its upper
// 128x128 tiles, as the full matrix in three bf16 planes (two launches).
void launch_f16x2_to_bf16x3(const SubView* views, const Sp2State* st, long long copy_stride, int n_sub, int max_rows,
                            uint8_t* arena, cudaStream_t s);
// out1 = a1 in + b1 I (kind 0), the SP2 start (kind 1) or its first-order change (kind 2) from
// the subgraph bounds; optional out2 = a2 in + b2 I.  Each output: master and / or planes
// (format nsplit).
void launch_affine_planes(const SubView* in, const SubView* out1, double a1, double b1, int master1, int nsplit1,
                          const SubView* out2, double a2, double b2, int master2, int nsplit2, int kind,
                          const double* bounds, int n_sub, int max_rows, uint8_t* arena, bool f64, cudaStream_t s);
// out1 = a1 E + b1 E^2 + c1 E^3 and out2 likewise (E, E^2, E^3 from masters), valid block only.
void launch_poly3(const SubView* e1, const SubView* e2, const SubView* e3, const SubView* out1, double a1, double b1,
                  double c1, int master1, int nsplit1, const SubView* out2, double a2, double b2, double c2,
                  int master2, int nsplit2, int n_sub, int max_rows, uint8_t* arena, bool f64, cudaStream_t s);
void launch_gershgorin(const SubView* views, int n_sub, int max_rows, const uint8_t* arena, double* lo, double* hi,
                       const long long* row_base, double* bounds, bool f64, cudaStream_t s);
void launch_sp2_replay_init(Sp2State* st, const double* bounds, const int* n_real, const int* steps, double mu, int n,
                            cudaStream_t s);
// Point every subgraph's buffer index (read by the *_from_sp2 operands) at copy `cur` and
// mark the recursion inactive (after the finite-temperature Fermi pass).
void launch_buffer_index(Sp2State* st, int cur, int n, cudaStream_t s);
void launch_sp2_init(Sp2State* st, const double* bounds, const int* n_real, double mu, double tol, int kmax, int n,
                     cudaStream_t s);
void launch_sp2_advance(Sp2State* st, const double* slots, const long long* tr_off, const int* n_diag,
                        int* n_active, int n, cudaStream_t s);

}  // namespace sedacs
