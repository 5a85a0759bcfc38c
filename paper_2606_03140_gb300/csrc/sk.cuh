// Slater-Koster model kernels: pair blocks, padded H/S gather, collected observables.
#pragma once
#include "common.cuh"

namespace sedacs {

struct SkGeom {
  double box[3];   // Angstrom
  int nimg[3];     // periodic images that can fall within r_off
};

void launch_pair_blocks(const ModelDev& m, const double* R, const int* species, const long long* pptr, const int* pcol,
                        int N, const SkGeom& g, void* h0b, void* sb, bool f64, cudaStream_t s);
void launch_loc_fill(const long long* sub_ptr, const int* sub_atoms, int* loc, int N, int n_sub, cudaStream_t s);
void launch_orb_offsets(const long long* sub_ptr, const int* sub_atoms, const int* species, const ModelDev& m,
                        int* orb_off, int* n_orb_sub, const int* n_core, int* n_core_orb, int n_sub, cudaStream_t s);
void launch_gather(const ModelDev& m, const long long* sub_ptr, const int* sub_atoms, const int* orb_off,
                   const int* species, const long long* pptr, const int* pcol, const void* h0b, const void* sb,
                   const int* loc, int N, const double* V, const long long* hoff, const long long* soff,
                   const int* n_pad, uint8_t* arena, int n_sub, const int* sub_of_row, long long total_rows,
                   int shift_only, bool f64, cudaStream_t s);
void launch_observables(const ModelDev& m, const double* R, const int* species, const SkGeom& g,
                        const long long* sub_ptr, const int* sub_atoms, const int* orb_off, const int* core_list,
                        const int* core_sub, const int* core_local, int n_core_total, const long long* pptr,
                        const int* pcol, const void* h0b, const void* sb, const int* loc, int N, const double* V,
                        const void* Dc, const void* Wc, const long long* dc_off, const long long* wc_off,
                        const int* n_pad, double* pop, double* eband, double* dU, int with_forces, bool f64,
                        cudaStream_t s);
void launch_gd(const ModelDev& m, const long long* sub_ptr, const int* sub_atoms, const int* orb_off,
               const int* species, const int* core_list, const int* core_sub, const int* core_local, int n_core_total,
               const void* Dc, bool f64, const long long* dc_off, const int* n_pad, const long long* gd_ptr, int* gd_col,
               double* gd_val, cudaStream_t s);
void launch_repulsion(const ModelDev& m, const double* R, const int* species, const SkGeom& g, const long long* pptr,
                      const int* pcol, int N, double* erep_atom, double* dU, bool f64, cudaStream_t s);

}  // namespace sedacs
