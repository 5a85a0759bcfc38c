/*
 * sedacs.h -- C ABI of the GB300 (sm_103a) engine for graph-based linear-scaling shadow QMD.
 *
 * The method is that of arxiv 2606.03140 ("SEDACS: A Scalable Framework for Complex
 * Chemistry Simulations"): an atom graph from a distance cutoff and the thresholded
 * atom-condensed density matrix (Sec. "Determining the Subgraphs", Sec. "Dynamic Graph
 * Adaption"), a core/halo partition (Fig. 1), a dense Fermi-operator solve on every
 * core+halo principal submatrix at one global chemical potential (Sec. "Matrix Functions
 * on a Graph", Eqs. 1-3), collection of the core rows into charges, energies and forces,
 * and extended-Lagrangian shadow Born-Oppenheimer dynamics of the charges (Sec. "Shadow
 * Molecular Dynamics", Eqs. NEQ/HW; SI Secs. B-C).  The electronic model is a synthetic sp
 * Slater-Koster SCC tight-binding model whose constants are passed in sedacs_model.
 *
 * Conventions (every entry point):
 *  - Units at the boundary: Angstrom, fs, amu, elementary charge, Hartree.
 *  - Arrays are caller-owned.  Pointers are HOST pointers unless device I/O is switched
 *    on with sedacs_set_device_io(), after which every array argument of the compute
 *    entry points is a DEVICE pointer (cudaMalloc / torch) read and written on the
 *    stream given there.
 *  - Positions R are row-major [N][3]; forces and velocities likewise.
 *  - Charges n, q are net Mulliken electron populations minus the valence count
 *    (electron excess, e) per atom.
 *  - Every call returns a sedacs_status; on failure sedacs_last_error() holds a message.
 *    No C++ exception crosses the boundary.  A context is not thread-safe.
 *  - The library allocates device memory inside the context; sedacs_destroy frees it.
 */
#ifndef SEDACS_H
#define SEDACS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sedacs_ctx sedacs_ctx;

typedef enum {
  SEDACS_OK = 0,
  SEDACS_EINVAL = 1,     /* bad argument or state */
  SEDACS_ENOMEM = 2,     /* device allocation failed */
  SEDACS_ECUDA = 3,      /* CUDA runtime error */
  SEDACS_ENOCONV = 4,    /* SCC did not converge within max_iter */
  SEDACS_ETIMEOUT = 5,   /* a bounded device wait gave up (kernel returned early) */
  SEDACS_ENUMERIC = 6,   /* NaN / Inf found in a result */
  SEDACS_EPRECISION = 7, /* the chemical potential of Eq. 2 was not found (no bracket / no convergence) */
  SEDACS_ECAPACITY = 8,  /* a fixed-size device buffer was too small */
  SEDACS_EIO = 9         /* a checkpoint file could not be written, opened or read */
} sedacs_status;

/* Synthetic sp Slater-Koster SCC-TB model (SI Sec. D).  Species 0 = H, 1 = C, 2 = O.
 * v0[i][j][X], X = ss sigma, sp sigma (s on i, p on j), pp sigma, pp pi (Hartree);
 * V_X(r) = v0 exp(-r/decay) sw(r), quintic switch sw from r_on to r_off (Angstrom);
 * overlap = overlap_scale * V / (1 Hartree); repulsion rep_a exp(-r/rep_decay) sw(r). */
typedef struct {
  int32_t n_orb[3];
  double eps_s[3], eps_p[3], hubbard_u[3], z_val[3], mass[3];
  double v0[3][3][4];
  double decay, overlap_scale, r_on, r_off;
  double rep_a[3][3];
  double rep_decay;
} sedacs_model;

/* Run parameters.  precision: 0 = plain FP64 on the CUDA cores; 1 = FP32-class on tcgen05
 * tensor cores with FP32 accumulation: the products of the Fermi-operator recursion (and the
 * T -> 0 SP2 squares) in the dual half-precision format of Finkelstein et al. (2021),
 * x = hi + 2^-11 lo in two fp16 planes (22 significant bits; three products hi*hi + hi*lo +
 * lo*hi), every other dense product with three-way bf16 splitting (24 bits, six products);
 * 4 = FP32-class with three-way bf16 splitting in every product; 2 = mixed BF16 (recursion
 * products with two-way bf16 splitting; S^-1/2 and the core-row back-transform three-way);
 * 3 = pure bf16 recursion products (diagnostic).  In 1-4 the Ewald sums run in FP32 with FP64
 * reductions; electron counts, energies and forces are summed in FP64.
 * kernel: 0 = K0 = -c_k0 I (SI Sec. B); 1 = preconditioned rank-m Krylov (SI Sec. B);
 * 2 = learned preconditioner (message-passing network, see sedacs_gnn_*), judged against 1. */
typedef struct {
  double r_graph;       /* distance-graph cutoff, Angstrom */
  double tau;           /* |D| threshold of the density graph */
  int32_t core_size;    /* target atoms per core (cores = round(N / core_size)) */
  int32_t precision;
  int32_t kernel;
  int32_t krylov_rank;  /* maximum rank m */
  double krylov_tol;    /* relative residual tolerance of the low-rank kernel */
  double c_k0;          /* K0 = -c I */
  double scc_tol;       /* max |q - n| for SCC convergence, e */
  double scc_alpha;     /* linear mixing coefficient */
  double sp2_tol;       /* SP2 stop: Tr(X - X^2) < sp2_tol * n_orbitals (0: 1e-7 in the mixed forms,
                           1e-9 in FP64) */
  int32_t sp2_kmax;     /* maximum SP2 steps */
  int32_t ns_iters;     /* Newton-Schulz steps for S^-1/2; 0: automatic (mixed forms: degree-6 Taylor
                           polynomial of (I + E)^-1/2 in three products when |s - I| <= 0.13 in
                           every subgraph, else 3 steps; FP64: 4 steps) */
  double ewald_tol;     /* relative accuracy of the Ewald sums (0: 1e-12 FP64, 1e-8 mixed) */
  int32_t judge_every;  /* kernel 2: every judge_every MD steps compare with the Krylov kernel */
  double judge_tol;     /* kernel 2: relative error above which the Krylov kernel takes over */
  double Te;            /* electronic temperature, K.  Te > 0: the Fermi operator of Eq. 2 at
                           beta = 1 / (k_B Te) by the recursive tanh-doubling expansion, and mu
                           from the collected count (Eq. 2: Tr[D S] = N_e).  Te = 0: the T -> 0
                           mu-branch SP2 recursion at a chemical potential the caller gives. */
  int32_t mu_given;     /* Te > 0: 1 = use the mu passed to the density calls as given (no Eq. 2 solve) */
  double fermi_lin;     /* Te > 0: after a Fermi pass at mu0 the count is brought to N_e by the mu step
                           dmu of its fourth-order expansion (D += sum_k (beta dmu)^k / k! D_k, with
                           d^kF/dmu^k = beta^k X_k: X_1 = s = F - F^2, X_2 = t = s (I - 2F),
                           X_3 = t (I - 2F) - 2 s^2, X_4 = X_3 (I - 2F) - 6 s t) when |beta dmu| is at
                           most this; otherwise another pass runs (0: 0.2 in the FP32-class forms,
                           1e-2 in FP64; remainder <= (beta dmu)^5 / 120 x 0.25 per occupation) */
  int32_t graph_rule;   /* graph from the previous density graph G^D: 0 = edge when the minimum-image
                           distance is below r_graph or G^D exceeds tau in either direction; 1 = the
                           weighted two-hop rule (Sec. "Dynamic Graph Adaption", Eq.
                           "Graph_Adaptation"): P = G^N G^D with G^N_IK = exp(-graph_alpha R_IK^2)
                           on the pairs with R^2 < ln(2 / tau) / graph_alpha (Angstrom) and
                           G^N_II = 1, edge when P_IJ or P_JI exceeds tau (r_graph unused).  Without
                           a density graph (first build) both use the distance rule.  A G^D row
                           holding more than ~1,500 distinct two-hop columns -> SEDACS_ECAPACITY. */
  double graph_alpha;   /* G^N decay, Angstrom^-2 (paper: 0.7) */
} sedacs_params;

/* Fill p with the defaults (r_graph 3.0, tau 1e-3, core_size 32, precision 1, kernel 0,
 * krylov_rank 4, krylov_tol 1e-2, c_k0 0.5, scc_tol 1e-8, scc_alpha 0.2, sp2_tol 0,
 * sp2_kmax 60, ns_iters 0, ewald_tol 0, judge_every 20, judge_tol 0.1, Te 300, mu_given 0,
 * fermi_lin 0, graph_rule 0, graph_alpha 0.7). */
void sedacs_default_params(sedacs_params* p);

/* Create a context for N atoms of the given species in an orthorhombic periodic box
 * (box > 2 * r_off on every axis is not required; box > r_off is).  Copies every input. */
sedacs_status sedacs_create(int32_t n_atoms, const int32_t* species, const double box[3], const sedacs_model* model,
                            const sedacs_params* params, sedacs_ctx** out);
void sedacs_destroy(sedacs_ctx* ctx);
const char* sedacs_last_error(const sedacs_ctx* ctx);

/* Replace the run parameters of a context (kernel, tolerances, graph cutoff, ...);
 * precision, core_size and ewald_tol must keep their creation values. */
sedacs_status sedacs_set_params(sedacs_ctx* ctx, const sedacs_params* params);

/* Device I/O: on != 0 makes every array argument a device pointer used on `stream`
 * (a cudaStream_t, may be 0 for the legacy default stream).  on = 0 restores host I/O. */
sedacs_status sedacs_set_device_io(sedacs_ctx* ctx, int32_t on, void* stream);

/* ---- a1: atom graph (Sec. "Determining the Subgraphs", Fig. 1a/e; Sec. "Dynamic Graph Adaption").
 * Edge (I,J), I != J, iff the minimum-image distance < r_graph or the density graph
 * value exceeds tau in either direction.  gd: optional CSR over atoms of the previous
 * atom-condensed density graph (ptr [N+1] int64, col int32, val double; NULL = none).
 * use_prev_D != 0 takes the density graph of the last sedacs_subgraph_density call instead.
 * A gd given here also serves the graph rebuilds of sedacs_scc_step / sedacs_xlbomd_init /
 * sedacs_xlbomd_step until the context has computed a density of its own (a ground state
 * handed over from another context keeps its graph).
 * The graph is kept in the context; *nnz receives its number of directed edges.
 * Integer result, bit-reproducible (separately rounded IEEE operations, no FMA). */
sedacs_status sedacs_graph_build(sedacs_ctx* ctx, const double* R, const int64_t* gd_ptr, const int32_t* gd_col,
                                 const double* gd_val, int64_t gd_nnz, int32_t use_prev_D, int64_t* nnz);
/* Copy the current graph out: row_ptr [N+1], col [nnz] (columns ascending per row). */
sedacs_status sedacs_graph_get(sedacs_ctx* ctx, int64_t* row_ptr, int32_t* col);

/* ---- a2: cores and halos (Fig. 1b/c).  Recursive coordinate bisection of the wrapped
 * positions into round(N/core_size) cores, then the one-hop halo of every core on the
 * current graph.  *n_parts receives the number of subgraphs. */
sedacs_status sedacs_partition(sedacs_ctx* ctx, const double* R, int32_t* n_parts);
/* Use caller-given cores (core_ptr [n_parts+1], core [N]; host or device arrays, read only)
 * instead of RCB, each core's atoms sorted on entry.  Every atom in exactly one core, every core
 * holding at least one atom (so n_parts <= N); otherwise SEDACS_EINVAL with the context's cores
 * unchanged.  With a graph present the halos are recomputed. */
sedacs_status sedacs_set_cores(sedacs_ctx* ctx, int32_t n_parts, const int64_t* core_ptr, const int32_t* core);
/* Recompute the halos of the current cores on the current graph. */
sedacs_status sedacs_update_halos(sedacs_ctx* ctx);
/* Sizes of the current subgraphs: *n_parts, total core atoms, total subgraph atoms. */
sedacs_status sedacs_parts_sizes(sedacs_ctx* ctx, int32_t* n_parts, int64_t* n_sub_atoms);
/* Subgraph atom lists: sub_ptr [n_parts+1], sub_atoms (core ascending then halo ascending),
 * n_core [n_parts] (core atoms lead every list). */
sedacs_status sedacs_parts_get(sedacs_ctx* ctx, int64_t* sub_ptr, int32_t* sub_atoms, int32_t* n_core);

/* ---- a3: Coulomb potential V = gamma b by Ewald summation (SI Sec. D), Hartree per e. */
sedacs_status sedacs_coulomb_potential(sedacs_ctx* ctx, const double* R, const double* b, double* V);

/* ---- a4-a9: graph-partitioned density (Eqs. 1-3) at trial charges n for the current
 * graph and subgraphs.  Per subgraph: gather h = H0 + 1/2 (S V + V S) and s, Z = s^-1/2,
 * h~ = Z h Z, the Fermi operator X = [exp(beta (h~ - mu I)) + I]^-1 (Eq. 2; Te > 0: recursive
 * tanh-doubling expansion on the tensor cores; Te = 0: the mu-branch SP2 recursion), core
 * rows D_c = 2 Z_c X Z and W_c = 2 Z_c X h~ Z; then Mulliken charges, band energy and the
 * density graph.  mu (Hartree): Te > 0: in = starting guess of the Eq. 2 solve (NaN: none),
 * out = the chemical potential whose collected count Tr[D S] equals N_e (with mu_given = 1:
 * used as given); Te = 0: used as given (NaN -> SEDACS_EINVAL).  No mu in the search bracket
 * -> SEDACS_EPRECISION.  q [N] out, e_band out (Hartree), sp2_iters [n_parts] out (nullable:
 * SP2 steps when Te = 0, else the tanh doublings of the last pass in every entry). */
sedacs_status sedacs_subgraph_density(sedacs_ctx* ctx, const double* R, const double* n, double* mu, double* q,
                                      double* e_band, int32_t* sp2_iters);
/* Net Mulliken charges q [N] (e) of the last density call (also after sedacs_xlbomd_step: the
 * density of the last step's positions and charges n). */
sedacs_status sedacs_charges(sedacs_ctx* ctx, double* q);
/* Energies of the last density call: e[0] band Tr[D H0], e[1] Coulomb 1/2 (2q - n)^T gamma n,
 * e[2] repulsion, e[3] total shadow potential (Hartree). */
sedacs_status sedacs_energy(sedacs_ctx* ctx, double* e);
/* ---- a10: forces of the last density call at fixed n (Eq. NEQ), Hartree/Angstrom [N][3]. */
sedacs_status sedacs_forces(sedacs_ctx* ctx, double* F);
/* Density graph of the last density call: sizes, then rows (core atom I: G^D_IJ over its subgraph). */
sedacs_status sedacs_density_graph_size(sedacs_ctx* ctx, int64_t* nnz);
sedacs_status sedacs_density_graph_get(sedacs_ctx* ctx, int64_t* ptr, int32_t* col, double* val);
/* Dense blocks of subgraph `part` from the last density call (row-major, n x n, FP64 copy):
 * which = 0 h, 1 s, 2 Z, 3 h~; core rows (n_core_orb x n): 4 D_c, 5 W_c.  *n, *n_core_orb out. */
sedacs_status sedacs_subgraph_matrix(sedacs_ctx* ctx, int32_t part, int32_t which, double* out, int32_t* n,
                                     int32_t* n_core_orb);

/* ---- a11: charge response dq/dn v (SI Sec. B, Eq. "dfdv") on the subgraphs of the last
 * density call.  Te > 0: canonical (mu moves so that the collected count stays N_e), by a
 * central difference of two density passes at n +- eps v (eps max|v| = 1e-3 e in the FP32-class
 * forms, 1e-4 e in FP64); the arena's h and h~ then hold the last perturbed pass.  Te = 0: at
 * fixed mu by first-order perturbation of the SP2 recursion. */
sedacs_status sedacs_charge_response(sedacs_ctx* ctx, const double* v, double* dq);
/* Kernel action u ~ K f = J^-1 f (SI Sec. B): K0 = -c I (kernel 0) or the preconditioned
 * rank-m Krylov approximation (kernel 1); *rank receives the rank used. */
sedacs_status sedacs_kernel_apply(sedacs_ctx* ctx, const double* f, double* u, int32_t* rank);

/* ---- a12: self-consistent charges (Sec. "Determining the Subgraphs", SI Sec. C).  Starting
 * from n (inout), iterates graph -> halos -> density -> n update until max |q - n| <= scc_tol
 * (linear mixing, or the kernel quasi-Newton step n <- n - K (q - n) once max |q - n| < 0.1 when
 * kernel = 1 (rank-m Krylov) or 2 (learned)).  Every density call solves Eq. 2 for mu (Te > 0),
 * starting from the previous iteration's value.
 * Cores must exist (sedacs_partition / sedacs_set_cores).  mu inout as in sedacs_subgraph_density. */
sedacs_status sedacs_scc_step(sedacs_ctx* ctx, const double* R, double* n, int32_t max_iter, double* mu,
                              double* resid_max, int32_t* iters);

/* ---- a12: XL-BOMD (Eqs. NEQ/HW; integrator of the paper's refs.: K = 5 dissipation,
 * kappa 1.82, alpha 0.018).  sedacs_xlbomd_init sets R, V (A/fs), the charge history n0
 * (normally the SCC solution) and mu, and evaluates forces.  sedacs_xlbomd_step advances
 * nsteps steps of dt_fs; R, V inout; energies [nsteps][3] (kinetic, shadow potential, total;
 * Hartree) out, nullable; n_out [N] (nullable) receives the final n. */
sedacs_status sedacs_xlbomd_init(sedacs_ctx* ctx, const double* R, const double* V, const double* n0, double mu);
sedacs_status sedacs_xlbomd_step(sedacs_ctx* ctx, double* R, double* V, int32_t nsteps, double dt_fs,
                                 double* energies, double* n_out);

/* ---- a13: learned charge-response preconditioner.  The paper names data-driven acceleration
 * as an extension (Sec. "Summary and Conclusions"); the network is this library's reading:
 * K_NN(y) = -c_k0 y + G(y), G a 3-layer, 64-wide message-passing network on the current atom
 * graph that is linear in y (species embedding times y, radial edge filters of the minimum-image
 * distance with a 6 A cosine cutoff, residual 64 x 64 mixes, linear read-out).  Parameters are a
 * flat FP64 vector of sedacs_gnn_num_params() entries (device copy in FP32): e[3][64], then per
 * layer C[8][64], A[64][64], B[64][64], then w[64].  Trained by Adam on pairs of the Krylov
 * kernel (SI Sec. B): with kernel 1 and collection on, every Krylov vector adds the pair
 * (x = J v, v) and every kernel application the pair (f, K_m f) to a ring of `capacity` pairs
 * (device memory). */
int32_t sedacs_gnn_num_params(void);
sedacs_status sedacs_gnn_init(sedacs_ctx* ctx, uint64_t seed);
sedacs_status sedacs_gnn_set_params(sedacs_ctx* ctx, const double* p);
/* grad != 0: the gradient of the last sedacs_gnn_param_grad call instead of the parameters. */
sedacs_status sedacs_gnn_get_params(sedacs_ctx* ctx, double* p, int32_t grad);
/* u = K_NN(y) on the current graph and positions. */
sedacs_status sedacs_gnn_apply(sedacs_ctx* ctx, const double* y, double* u);
/* grad = d/dp sum_i gu_i K_NN(y)_i (host or device arrays as the I/O mode says). */
sedacs_status sedacs_gnn_param_grad(sedacs_ctx* ctx, const double* y, const double* gu, double* grad);
sedacs_status sedacs_gnn_collect(sedacs_ctx* ctx, int32_t on, int32_t capacity);
/* Adam (lr) for `epochs` full-batch steps on the mean of |K_NN(x) - v|^2 over the given pairs
 * (X, V: [n_pairs][N]) or, with X = NULL, over the collected pairs.  Losses of the first and
 * the last step out. */
sedacs_status sedacs_gnn_train(sedacs_ctx* ctx, const double* X, const double* V, int32_t n_pairs, int32_t epochs,
                               double lr, double* loss_first, double* loss_last);
/* Last judged relative error |K_NN f - K_m f| / |K_m f| and the number of fallbacks to the
 * Krylov kernel during XL-BOMD with kernel 2. */
sedacs_status sedacs_kernel_judge(sedacs_ctx* ctx, double* last_error, int32_t* fallbacks);

/* Diagnostics of the last density call (Te > 0): info[0] collected electron count minus N_e
 * after the mu solve, info[1] dN/dmu at the accepted pass (e/Ha), info[2] the linear mu step
 * applied after it (Ha), info[3] Fermi-operator evaluations, info[4] tanh doublings per pass, info[5]
 * evaluations that shifted mu at the stage kept by a full pass instead of running one, then per
 * evaluation the triple (mu, N_e - N(mu), dN/dmu) (zeros past the last).  n_info entries are written. */
sedacs_status sedacs_density_info(sedacs_ctx* ctx, double* info, int32_t n_info);

/* Wall time (ms, CUDA events on the context stream) of the phases of the last call:
 * t[0] graph+halos, t[1] Coulomb, t[2] gather, t[3] S^-1/2 + h~, t[4] Fermi operator, t[5] collect,
 * t[6] forces, t[7] kernel + update.  Also the number of kernels launched since the last
 * sedacs_reset_counters() in *launches. */
sedacs_status sedacs_phase_times(sedacs_ctx* ctx, double* t, int64_t* launches);
sedacs_status sedacs_reset_counters(sedacs_ctx* ctx);
/* Per-launch timing of the Fermi-operator products (Te > 0: the tanh-doubling recursion; Te = 0:
 * the SP2 squares): on != 0 records CUDA events around every launch on the context stream.
 * Returns the accumulated kernel time (ms), number of launches and the algorithmic work of
 * those launches in flops, counting a symmetric product of two n x n matrices (upper triangle)
 * as n^3 (n the orbital count of the subgraph), since the last reset. */
sedacs_status sedacs_kernel_stats(sedacs_ctx* ctx, int32_t on, double* sp2_ms, int64_t* sp2_launches,
                                  double* sp2_flops);
/* The part of those statistics from the products in two fp16 planes (the recursion of the
 * FP32-class form 1), with their algorithmic DRAM bytes: over the upper triangle of every
 * n x n subgraph (n (n + 1) / 2 elements), the operands read once (4 bytes an element; one read
 * when both operands are the same matrix), each FP32 addend (4), the output planes (4, or 6 in
 * three bf16 planes), the FP32 master (4) unless the product keeps planes only, and a second
 * output (4).  Outputs are host scalars; counters as for sedacs_kernel_stats. */
sedacs_status sedacs_kernel_stats_fp16(sedacs_ctx* ctx, double* ms, int64_t* launches, double* flops,
                                       double* bytes);

/* Assignment of whole subgraphs to n_ranks ranks for a step sharded over several GPUs (host
 * only; needs no context and no GPU).  The subgraph solves are independent, with a cost that grows
 * as the cube of the orbital count (Sec. "Scalability"); the caller passes one cost per subgraph
 * (host array, >= 0 and finite; n_i^3 for the subgraph solves).  LPT (Graham 1969): subgraphs in
 * descending cost, equal costs by ascending index, each to the rank with the least load so far,
 * equal loads to the lowest rank; the largest load is within 4/3 - 1/(3 n_ranks) of the optimum.
 * owner[n_sub] receives each subgraph's rank, rank_load[n_ranks] each rank's summed cost (host
 * arrays, caller-owned).  n_sub < 0, n_ranks <= 0, a null array or a negative or non-finite cost
 * -> SEDACS_EINVAL. */
sedacs_status sedacs_shard_lpt(int32_t n_sub, const double* cost, int32_t n_ranks, int32_t* owner,
                               double* rank_load);

/* Core refinement for the tiles of the subgraph solves (not in the paper, which notes that a
 * subgraph's cost grows with the cube of its size).  The tensor-core products work on 128-orbital
 * tiles, so a subgraph of n orbitals (core + halo) costs about T^3, T = ceil(n / 128).  Single core
 * atoms move to an adjacent core (a graph neighbour's core) while that lowers the integer score
 * sum over subgraphs of 128000 T^3 + (n - 128 (T - 1)) (T^3 - (T - 1)^3); cores more than 48
 * orbitals above their boundary are left alone and every core keeps at least min_core atoms.
 * Deterministic: cores by index, each core's atoms ascending (a snapshot taken at its turn),
 * target cores ascending, the first best strict improvement; at most `rounds` passes, fewer when a
 * pass moves nothing.  Uses the current graph and cores (sedacs_graph_build, sedacs_partition
 * first: SEDACS_EINVAL otherwise), sets the new cores and recomputes the halos.  score_before /
 * score_after (host, nullable) receive the score. */
sedacs_status sedacs_refine_cores(sedacs_ctx* ctx, int32_t rounds, int32_t min_core, int64_t* score_before,
                                  int64_t* score_after);

/* Self-test of the bounded device waits (the paper has no counterpart): one device thread waits on
 * a flag that nothing sets, gives up after about limit_us microseconds (1 .. 1,000,000) of SM
 * cycles and raises the timeout bit every bounded wait of the library raises.  Returns
 * SEDACS_ETIMEOUT (SEDACS_EINVAL for a limit out of range); the bit is cleared as it is reported,
 * and the context stays usable. */
sedacs_status sedacs_selftest_wait(sedacs_ctx* ctx, int32_t limit_us);

/* ---- Checkpoint of the XL-BOMD state.  sedacs_checkpoint_save writes to the file `path` the
 * state a shadow-dynamics step continues from (Eqs. NEQ / HW): positions, velocities and forces,
 * the dynamical charges n, the charges q of the last density, the six-deep history of n of the
 * dissipative integrator with its head, the step count, mu and the mu of the step before, the
 * atom-condensed density graph the next graph is built from, and the core lists; the context
 * must have run sedacs_xlbomd_init (SEDACS_EINVAL otherwise).  sedacs_checkpoint_load restores
 * that state into a context created with the same atoms, model and parameters (the atom count,
 * precision form and Te are checked: SEDACS_EINVAL); the next sedacs_xlbomd_step then continues
 * the trajectory (the R and V it is given are outputs only).  A missing, truncated or foreign
 * file -> SEDACS_EIO.  The learned preconditioner's parameters are not included (they are read
 * and set with sedacs_gnn_get_params / sedacs_gnn_set_params).  The paper has no counterpart
 * beyond the restart files of its MD driver. */
sedacs_status sedacs_checkpoint_save(sedacs_ctx* ctx, const char* path);
sedacs_status sedacs_checkpoint_load(sedacs_ctx* ctx, const char* path);

/* ---- Allocation-free distance graph.  The paper has no counterpart to this entry point;
 * it exists for callers that cannot allocate device memory at the time of the call (programs
 * whose device memory belongs to another allocator, loops that cannot take cudaMalloc's
 * implicit synchronisation).  It writes the
 * distance part of the graph of sedacs_graph_build (edge iff minimum-image distance
 * < r_graph, columns ascending, bit-identical) into caller-owned DEVICE arrays: R [N][3]
 * (Angstrom), row_ptr [N+1], col [col_capacity]; *nnz (host) receives the edge count.
 * No context, no cudaMalloc / cudaFree: the scratch is a fixed array inside the library
 * (N <= 16384 atoms; larger N -> SEDACS_EINVAL), present on every GPU that loaded the
 * library until exit; the first call on a device looks up that array's address.  The call
 * copies the edge count to the host and synchronises `stream`, so it cannot be recorded
 * into a CUDA graph.  Every call shares the one array: calls that can overlap
 * on the GPU (other streams, other host threads) race and must be serialised by the
 * caller.  col too small -> SEDACS_ECAPACITY with *nnz = the size needed (col untouched).
 * A CUDA error already pending when the call starts -> SEDACS_ECUDA, left pending for the
 * caller.  Runs on `stream` (cudaStream_t) and returns after it has finished. */
sedacs_status sedacs_graph_build_noalloc(const double* R, int32_t n_atoms, const double box[3], double r_graph,
                                         int64_t* row_ptr, int32_t* col, int64_t col_capacity, int64_t* nnz,
                                         void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SEDACS_H */
