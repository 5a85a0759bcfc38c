// Ewald summation of the periodic Gaussian-gamma Coulomb interaction on the GPU.
#pragma once
#include "common.cuh"

namespace sedacs {

struct EwaldGeom {
  double box_b[3];      // box in bohr
  double vol;           // bohr^3
  double eta;           // splitting parameter (1/bohr)
  double rc_b;          // real-space cutoff (bohr)
  double a[3][3];       // Gaussian screening a_IJ per species pair
  double u[3];          // Hubbard U per species
  int nmax[3];          // largest |m| per axis in reciprocal space
  int nmax_all;
  int nimg[3];          // periodic images needed in real space (small boxes)
  int nc[3];            // cell grid (cells at least rc wide)
  int brute;            // 1: loop over all atoms and images
};

struct KRow {           // reciprocal vectors with fixed (m1, m2), m3 in [m3lo, m3hi]
  int m1, m2, m3lo, m3hi;
  long long koff;       // index of (m1, m2, m3lo) in the flat k list
};

struct Ewald {
  static constexpr int kChunk = 1024;
  static constexpr int kRowChunks = 24;    // k-row chunks of the per-atom reciprocal sums
  EwaldGeom g{};
  int N_ = 0;
  bool fp64_ = true;
  int nrows_ = 0, nchunk_ = 0, m3max_ = 0;
  long long nk_ = 0;
  KRow* rows_d = nullptr;
  double* wk_d = nullptr;
  void* tab = nullptr;       // phase tables (float2 or double2)
  double* part = nullptr;    // structure-factor partial sums
  void* ws = nullptr;        // w(k) S(k)
  double* real_buf = nullptr;
  double* recip_buf = nullptr;
  double* rpart = nullptr;   // per-row-chunk partial sums
  double* scal = nullptr;
  int *cell_of = nullptr, *cell_count = nullptr, *cell_start = nullptr, *cell_atoms = nullptr;
  void* pos_s = nullptr;     // cell-sorted cell-relative coordinates and species (float4 / double4)
  int sb_tag_ = 0;           // tag of the charges whose S(k) sits in vector 0 of ws (0: none)
  const double* dR_ = nullptr;
  const int* dspecies_ = nullptr;
  ~Ewald();
  void release();
  // Parameters for relative accuracy ~tol; fp64 selects the arithmetic of the sums.
  cudaError_t setup(int N, const double box_A[3], const double hubbard_u[3], bool fp64, double tol);
  // Phase tables and cell list for positions dR (Angstrom, device, N x 3).
  cudaError_t prepare(const double* dR, const int* dspecies, cudaStream_t s);
  // V = gamma b (Ha per e).  A nonzero tag names b: a later gradient with the same tag and the
  // same b reuses its structure factor (valid until the next prepare or potential call).
  cudaError_t potential(const double* b, double* V, cudaStream_t s, int tag = 0);
  // G = d/dR (a^T gamma b) in Ha/A.
  cudaError_t gradient(const double* a, const double* b, double* G, cudaStream_t s, int tag = 0);
};

}  // namespace sedacs
