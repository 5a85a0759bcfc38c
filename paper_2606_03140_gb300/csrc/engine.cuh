// Host engine behind the C ABI: owns device buffers, the per-subgraph arena layout, the
// batched GEMM tables and the stream; runs the pipeline of the graph-partitioned solve.
#pragma once
#include <string>
#include <tuple>
#include <limits>
#include <vector>

#include "../../include/sedacs.h"
#include "dense.cuh"
#include "dense_ops.cuh"
#include "ewald.cuh"
#include "graph.cuh"
#include "sk.cuh"

namespace sedacs {

// A matrix slot of the arena: one matrix per subgraph (square n_pad x n_pad or core rows
// m_pad x n_pad), a row-major master (fp32 or fp64) and optionally three bf16 planes.
struct Slot {
  long long base = 0;        // byte offset of copy 0
  long long copy_stride = 0; // bytes between copies (ping-pong)
  long long master_bytes = 0;
  long long plane_stride = 0;
  bool rows = false;
  bool planes = false;
  int copies = 1;
};

enum SlotId : int {
  kS = 0, kH, kT, kY0, kY1, kZ0, kZ1, kP, kHt, kX, kT1, kDc, kT2, kWc,
  kR1, kR2,            // response: X dX, and dX (ping-pong)
  kdH, kdHt, kdT1, kdDc,
  kdT2, kdDt,          // core rows of t = s (I - 2F) (second-order mu term): Z_c t, 2 Z_c t Z
  kdT3, kdDu,          // core rows of the third-order term u: Z_c u, 2 Z_c u Z
  kdT4, kdDw,          // core rows of the fourth-order term w: Z_c w, 2 Z_c w Z
  kNumSlots
};

struct GemmOp {
  GemmMat* mats_d = nullptr;
  GemmWork* work_d = nullptr;
  int n_work = 0;
  double alpha = 1.0, beta = 0.0, g1 = 0.0, g2 = 0.0, alpha2 = 0.0;
  int mode = kModeGeneric;
  bool sym = false;          // symmetric output: upper tiles only (counted as n^3 flops)
  int ops_upper = 0;         // operands stored as upper tiles (fp16 two-plane path)
  int store_upper = 0;       // result stored as upper tiles (no mirror)
  int no_master = 0;         // fp16 two-plane path: result kept as planes only (no FP32 master)
  int same_ab = 0;           // A and B are one matrix (read once)
  int n_addends = 0;         // C1 / C2 added in the epilogue (FP32 masters)
  int dual = 0;              // second output (planes)
};

enum OpId : int {
  OP_NS_Y1 = 0,
  OP_NS_T0, OP_NS_T1, OP_NS_Y0, OP_NS_Y1b, OP_NS_Z0, OP_NS_Z1,
  OP_P0, OP_P1, OP_HT0, OP_HT1,
  OP_SP2,
  OP_T1_0, OP_T1_1, OP_DC0, OP_DC1, OP_T2, OP_WC0, OP_WC1,
  // response (first-order SP2), see response.cu
  OP_RSP_A, OP_RSP_B, OP_DP0, OP_DP1, OP_DHT0, OP_DHT1, OP_DT1_0, OP_DT1_1, OP_DDC0, OP_DDC1,
  // Z = s^-1/2 by the degree-6 Taylor polynomial of (I + E)^-1/2 (Paterson-Stockmeyer)
  OP_TE2, OP_TE3, OP_TZ,
  // finite-temperature Fermi operator (engine.cu, run_fermi): start U0 = tanh(z) = z q(z^2)
  // (Z2 = z z, Z4 = Z2 Z2, Horner in Z4), doublings U <- 2 U r(U^2) (V = U U, V2 = V V, Horner
  // in V2), the last doubling writing F = (I + U) / 2, and s = F - F^2
  OP_F_Z2, OP_F_Z4, OP_F_ST1, OP_F_SH0, OP_F_SH1, OP_F_SH2, OP_F_SH3, OP_F_U0_0, OP_F_U0_1,
  OP_F_V_0, OP_F_V_1, OP_F_V2, OP_F_IT1, OP_F_IH0, OP_F_IH1, OP_F_IH2, OP_F_IH3, OP_F_IH4, OP_F_IH5,
  OP_F_UP_0, OP_F_UP_1, OP_F_FIN, OP_F_S,
  // core rows of F into the response slots (dT1 = Z_c F), and W of s: T2 = dT1 h~, Ws = 2 T2 Z
  OP_F_FT1_0, OP_F_FT1_1, OP_F_T2S, OP_F_WS0, OP_F_WS1,
  // second-order mu term: t = s - 2 s F (kR1 copy 1), its core rows (kdT2, kdDt), T2 = kdT2 h~
  OP_F_T, OP_F_TT1_0, OP_F_TT1_1, OP_F_DT0, OP_F_DT1, OP_F_T2T,
  // mu shift at a saved doubling stage: U' = U Q + tau Q, Q ~ (I + tau U)^-1 (U in kY0), into kX
  OP_F_MOB_0, OP_F_MOB_1,
  // degree-9 inverse in powers of V^3 (fp16 two-plane form): [V^3 | T_1] from one product V V^2 (two
  // outputs), T_2 = V^3 T_1 + B_1, r = V^3 T_2 + B_0
  OP_F_I3, OP_F_I4, OP_F_I5,
  // third- and fourth-order mu terms: P = t F (kT), u = t - 2 P - 2 s s (kY0), its core rows
  // (kdT3, kdDu), T2 = kdT3 h~; Q = u F (kT), w = u - 2 Q - 6 s t (kY1), rows (kdT4, kdDw), T2
  OP_F_TF, OP_F_U, OP_F_UT1_0, OP_F_UT1_1, OP_F_DU0, OP_F_DU1, OP_F_T2U,
  OP_F_UF, OP_F_W, OP_F_WT1_0, OP_F_WT1_1, OP_F_DW0, OP_F_DW1, OP_F_T2W,
  // G = (I - V) r(V) from the last doubling (kT); s = F - F^2 = G^2 / 4 (OP_F_S)
  OP_F_G,
  OP_NUM
};

// Learned preconditioner (gnn.cu): parameters, Adam moments, activations, training pairs.
struct GnnState {
  float *P = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *act = nullptr, *part = nullptr, *ebas = nullptr;
  long long ebas_cap = 0;
  int nchunk = 0;
  int t = 0;                 // Adam step count
  double *gu = nullptr, *u = nullptr;
  bool collect = false;      // store (J v, v) pairs produced by the Krylov kernel
  double *pX = nullptr, *pV = nullptr;
  int pairs = 0, pair_cap = 0, pair_head = 0;
  int fallbacks = 0;         // judge decisions that returned to the Krylov kernel
  double last_judge = -1.0;  // last relative error |K_NN f - K_m f| / |K_m f|
};

struct Layout {
  int n_sub = 0;
  std::vector<int> n_real, n_pad, m_pad, n_core_orb, n_core_atoms, n_atoms;
  std::vector<long long> sq_off, rw_off;   // element offsets in square / rows slots
  long long sq_total = 0, rw_total = 0;
  int max_npad = 0, max_mpad = 0;
  long long tr_total = 0;
  std::vector<long long> tr_off;
  std::vector<int> n_diag;
};

int gnn_num_params();
}  // namespace sedacs

#include <unordered_map>

struct sedacs_ctx {
  // capacities of grow-only device buffers, keyed by the address of their pointer
  std::unordered_map<void**, size_t> caps;
  // system
  int N = 0;
  std::vector<int> species_h;
  double box[3] = {0, 0, 0};
  sedacs::ModelDev model{};
  sedacs_params prm{};
  double n_electrons = 0.0;
  cudaStream_t stream = 0;
  bool dev_io = false;
  std::string err;
  bool f64 = false;
  int tile = 128;
  int nsplit_sp2 = 3, nsplit_ns = 3;
  int nsplit_rsp = 3;    // plane format of the first-order SP2 replay (X and dX): fp16 two-plane
                         // SP2 forms replay in three bf16 planes (dX can exceed the fp16 range)
  int nsplit_fermi = 3;  // plane format of the finite-temperature Fermi recursion's products
  // finite-temperature Fermi operator: degrees of its two polynomials (kTanh*, kInv*), the
  // tanh doublings of the last pass, and the diagnostics of the last density call
  int fermi_j = 3, fermi_m = 4;   // Horner lengths (start: Z4 steps; inverse: V2 steps)
  bool fermi_v3 = false;          // inverse by the V^3-stride scheme with the two-output product
  int fermi_n = 0;                // doublings of the last pass
  double fermi_count_err = 0.0;   // collected count minus N_e after the mu solve
  double fermi_dndmu = 0.0;       // dN/dmu at the accepted pass (e / Ha)
  double fermi_dmu = 0.0;         // mu step applied (to second order) after the accepted pass
  double mu_prev = std::numeric_limits<double>::quiet_NaN();   // mu of the MD step before (predictor)
  int fermi_passes = 0;           // Fermi-operator passes of the last density call
  std::vector<double> fermi_hist; // per pass: mu, N_e - N(mu), dN/dmu
  // the stage of the last full pass kept for mu shifts (U_j in kR2 copy 1): its mu, its stage j
  // (doublings done) and the pass's doubling count; j < 0: none
  double fermi_saved_mu = 0.0;
  int fermi_saved_j = -1, fermi_saved_nd = 0;
  int fermi_reentries = 0;        // mu shifts at the saved stage in the last density call
  double sum_n3 = 0.0;            // sum over subgraphs of n_real^3 (flops of one symmetric product)
  bool ht_stale = false;          // h, h~ of the arena hold a perturbed state (response passes)
  double* d_rsp = nullptr;        // 8 N-vectors of the finite-difference response
  // device vectors
  int* d_err = nullptr;
  int* d_species = nullptr;
  double *d_R = nullptr, *d_n = nullptr, *d_q = nullptr, *d_V = nullptr, *d_pop = nullptr, *d_eband = nullptr;
  double *d_dU = nullptr, *d_F = nullptr, *d_erep = nullptr, *d_tmp = nullptr, *d_tmp2 = nullptr, *d_scal = nullptr;
  double *d_vel = nullptr, *d_hist = nullptr, *d_mass = nullptr, *d_zval = nullptr;
  double* d_vec = nullptr;   // scratch N-vectors for the kernel (Krylov)
  // graph
  sedacs::GraphBuilder gb, pb;
  long long* d_row_ptr = nullptr;
  int* d_col = nullptr;
  long long col_cap = 0, nnz = 0;
  bool have_graph = false;
  // pair list within r_off and its SK blocks
  long long* d_pptr = nullptr;
  int* d_pcol = nullptr;
  long long pcol_cap = 0, pnnz = 0;
  void *d_h0b = nullptr, *d_sb = nullptr;
  long long blk_cap = 0;
  bool pairs_valid = false;
  // density graph of the last density call
  long long* d_gd_ptr = nullptr;
  int* d_gd_col = nullptr;
  double* d_gd_val = nullptr;
  long long gd_cap = 0, gd_nnz = 0;
  bool have_gd = false;
  // external density graph uploaded by the caller
  long long* d_xgd_ptr = nullptr;
  int* d_xgd_col = nullptr;
  double* d_xgd_val = nullptr;
  long long xgd_cap = 0;
  // partition
  sedacs::Partitioner part;
  bool have_cores = false, have_subs = false;
  long long* d_sub_ptr = nullptr;
  int* d_sub_atoms = nullptr;
  long long sub_cap = 0;
  std::vector<long long> sub_ptr_h;
  std::vector<int> sub_atoms_h;
  int *d_orb_off = nullptr, *d_n_orb_sub = nullptr, *d_n_core = nullptr, *d_n_core_orb = nullptr;
  int *d_sub_of_row = nullptr, *d_core_sub = nullptr, *d_core_local = nullptr, *d_loc = nullptr;
  long long loc_cap = 0, rows_cap = 0;
  int n_core_total = 0;
  // layout and arena
  sedacs::Layout lay;
  sedacs::Slot slot[sedacs::kNumSlots];
  uint8_t* arena = nullptr;
  size_t arena_cap = 0;
  sedacs::GemmOp ops[sedacs::OP_NUM];
  sedacs::SubView* d_views[sedacs::kNumSlots] = {};
  sedacs::SubView* d_views_x1 = nullptr;   // X copy 1
  long long *d_hoff = nullptr, *d_soff = nullptr, *d_dcoff = nullptr, *d_wcoff = nullptr, *d_rowbase = nullptr;
  long long* d_tr_off = nullptr;
  int *d_n_pad = nullptr, *d_n_real = nullptr, *d_n_diag = nullptr;
  double *d_glo = nullptr, *d_ghi = nullptr, *d_bounds = nullptr, *d_slots = nullptr;
  sedacs::Sp2State* d_sp2 = nullptr;
  int* d_nactive = nullptr;
  long long* d_dcoff_d = nullptr;   // core-row offsets of the response density
  long long* d_dcoff_t = nullptr;   // core-row offsets of the second-order mu term (kdDt)
  long long* d_dcoff_u = nullptr;   // ... of the third-order term (kdDu)
  long long* d_dcoff_w = nullptr;   // ... of the fourth-order term (kdDw)
  double* d_dqpop = nullptr;        // response populations scratch
  long long* d_dhoff = nullptr;     // per-subgraph offsets of the response Hamiltonian
  int* d_steps = nullptr;           // SP2 step counts of the last density call
  std::vector<double> bounds_h;
  int zc = 0;              // Z buffer holding s^-1/2
  bool z_valid = false;
  bool geom_valid = false; // pair blocks / Ewald tables match d_R
  // Ewald
  sedacs::Ewald ew;
  bool ew_ready = false;
  // state of the last density call
  double mu = 0.0;
  bool have_density = false;
  std::vector<int> sp2_iters_h;
  double e_band = 0, e_coul = 0, e_rep = 0;
  bool have_forces = false;
  // learned preconditioner
  sedacs::GnnState gnn;
  // MD
  bool md_ready = false;
  long long md_step = 0;
  int hist_head = 0;
  // timing of the SP2 square kernel (per launch, events on the context stream)
  bool kstats = false;
  std::vector<cudaEvent_t> kev;
  // SP2 step control: per-step active counts copied into pinned host memory, one event per
  // step, so that the host waits on a step a few launches back instead of draining the stream
  bool have_xgd = false;  // a density graph was given to sedacs_graph_build (d_xgd_*)
  // Layout uploads staged in one host buffer and sent from pinned memory in one go
  // (rebuild_layout): (device destination, offset in stage_host, bytes)
  std::vector<uint8_t> stage_host;
  std::vector<std::tuple<void*, size_t, size_t>> stage_recs;
  uint8_t* stage_pinned = nullptr;
  size_t stage_pinned_cap = 0;
  bool fuse_forces = false;  // the next density's observables pass also contracts the forces
  bool du_ready = false;     // d_dU holds the band-structure force terms of the last density
  int ew_tag = 0;         // tag of the Coulomb potential of d_n at the current geometry
  int* h_nactive = nullptr;        // mapped pinned: active subgraphs after each SP2 step
  int* h_nactive_dev = nullptr;    // its device alias
  int h_nactive_cap = 0;
  std::vector<cudaEvent_t> sp2_ev;
  int kev_used = 0;
  double k_ms = 0.0, k_flops = 0.0;
  long long k_launches = 0;
  // the same for the fp16 two-plane products alone, with their algorithmic bytes
  std::vector<double> kev_bytes;   // per recorded launch: bytes (fp16 launches), -1 otherwise
  double k16_ms = 0.0, k16_flops = 0.0, k16_bytes = 0.0;
  long long k16_launches = 0;
  double sum_tri = 0.0;            // sum over subgraphs of n (n + 1) / 2
  // timing
  cudaEvent_t ev[10] = {};
  double t_phase[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long launches = 0;
};
