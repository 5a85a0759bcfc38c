// Graph construction, partition and halo builders (device memory owned by the builder).
#pragma once
#include <vector>
#include "common.cuh"

namespace sedacs {

struct RcbSeg {
  int start;            // first position in the permutation
  int count;            // atoms in the segment
  long long scratch;    // offset of its sort scratch
};

struct GraphBuilder {
  int* cell_of = nullptr;
  int* cell_count = nullptr;
  int* cell_start = nullptr;
  int* cell_fill = nullptr;
  int* cell_atoms = nullptr;
  int* cnt = nullptr;
  int* fillc = nullptr;
  int* ucnt = nullptr;
  long long* cptr = nullptr;
  int* cand = nullptr;
  int cap_n = 0, cap_cells = 0;
  long long cap_cand = 0;
  // weighted two-hop rule: neighbour rows (G^N) and the thresholded entries of P = G^N G^D
  int* n_cnt = nullptr;
  long long* n_ptr = nullptr;
  int* n_col = nullptr;
  int* p_cnt = nullptr;
  long long* p_ptr = nullptr;
  int* p_col = nullptr;
  double* p_val = nullptr;
  long long cap_ncol = 0, cap_p = 0;
  ~GraphBuilder();
  void release();
  // Builds the symmetric CSR of the atom graph into row_ptr (device, N+1) and *col_out
  // (device, grown as needed).  gptr/gcol/gval: optional device CSR of the previous
  // atom-condensed density graph.  keep_prev: the graph already in row_ptr / *col_out keeps all
  // its edges (the new graph is its union with the rule's edges).  rule 0: distance below r_graph
  // or density-graph entry above tau; rule 1 (with a density graph): the weighted two-hop rule,
  // edge when P_IJ or P_JI exceeds tau, P = G^N G^D, G^N_IK = exp(-alpha R_IK^2) on the pairs with
  // R^2 < ln(2 / tau) / alpha and G^N_II = 1 (each G^D row must list a column once).
  cudaError_t build(const double* dR, int N, const double box[3], double r_graph, const long long* gptr,
                    const int* gcol, const double* gval, double tau, long long* row_ptr, int** col_out,
                    long long* col_cap, long long* nnz_host, int* derr, cudaStream_t s, bool exact = true,
                    bool keep_prev = false, int rule = 0, double alpha = 0.7);
};

struct Partitioner {
  int* perm = nullptr;        // atoms grouped by core, each core ascending
  double* skey = nullptr;
  int* sidx = nullptr;
  RcbSeg* segs_d = nullptr;
  unsigned* bits = nullptr;
  int* hcnt = nullptr;
  int cap_n = 0, cap_seg = 0, cap_hcnt = 0, cap_subptr = 0;
  long long cap_scr = 0, cap_bits = 0;
  int n_parts = 0;
  std::vector<RcbSeg> leaves;       // core segments in perm (host copy)
  std::vector<int> halo_count_h;
  ~Partitioner();
  void release();
  cudaError_t rcb(const double* dR, int N, const double box[3], int core_size, cudaStream_t s);
  cudaError_t set_cores(const std::vector<std::vector<int>>& cores, int N, cudaStream_t s);
  // Halos of the current cores on graph (row_ptr, col); writes the subgraph atom lists.
  cudaError_t halos(const long long* row_ptr, const int* col, int N, long long** sub_ptr_d, int** sub_atoms_d,
                    long long* sub_cap, std::vector<long long>& sub_ptr_h, cudaStream_t s);
};

}  // namespace sedacs
