// Allocation-free build of the distance graph.
//
// Some callers cannot allocate device memory when they call into this library: programs
// whose device memory is owned by another allocator or memory pool that must not be
// bypassed, and loops that cannot afford the implicit device synchronisation of
// cudaMalloc / cudaFree.  sedacs_graph_build_noalloc serves them: it
// writes the same CSR as the distance part of sedacs_graph_build into arrays the caller
// owns and allocates nothing.  Its scratch (one neighbour count per atom and a status word)
// is a file-scope __device__ array, present on every GPU that loads the library until the
// process exits.  Host code cannot use that symbol as a device address, so on the first
// call on each device the address is looked up with cudaGetSymbolAddress and cached.
#include <mutex>

#include "../../include/sedacs.h"
#include "common.cuh"

namespace {

constexpr int kNoAllocMaxAtoms = 16384;
constexpr int kNoAllocMaxDevices = 64;

// counts[0 .. kNoAllocMaxAtoms), then one status word.
static __device__ __align__(256) int g_noalloc_scratch[kNoAllocMaxAtoms + 1];

int* g_scratch_addr[kNoAllocMaxDevices] = {};
std::mutex g_scratch_mutex;

struct Box3 {
  double L[3];
};

__device__ __forceinline__ double na_r2(const double* R, int i, int j, const Box3& b) {
  double d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double dx = __dsub_rn(R[3 * j + a], R[3 * i + a]);
    d[a] = __dsub_rn(dx, __dmul_rn(b.L[a], rint(__ddiv_rn(dx, b.L[a]))));
  }
  return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

__global__ void na_count(const double* R, int N, Box3 b, double rg2, int* cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int c = 0;
  for (int j = 0; j < N; ++j)
    if (j != i && na_r2(R, i, j, b) < rg2) ++c;
  cnt[i] = c;
}

// Exclusive scan into the caller's row_ptr (single CTA).  It always writes status[0] (1 when col
// is too small, else 0), so the status word needs no clearing between calls; na_count writes
// every count it reads.
__global__ void na_scan(const int* cnt, int N, long long* row_ptr, int* status, long long cap) {
  __shared__ long long part[1024];
  const int per = (N + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per, b1 = min(N, b0 + per);
  long long s = 0;
  for (int i = b0; i < b1; ++i) s += cnt[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long acc = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const long long v = part[t];
      part[t] = acc;
      acc += v;
    }
    row_ptr[N] = acc;
    status[0] = acc > cap ? 1 : 0;
  }
  __syncthreads();
  long long acc = part[threadIdx.x];
  for (int i = b0; i < b1; ++i) {
    row_ptr[i] = acc;
    acc += cnt[i];
  }
}

__global__ void na_fill(const double* R, int N, Box3 b, double rg2, const long long* row_ptr, int* col,
                        const int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || status[0] != 0) return;
  long long p = row_ptr[i];
  for (int j = 0; j < N; ++j)
    if (j != i && na_r2(R, i, j, b) < rg2) col[p++] = j;
}

}  // namespace

extern "C" sedacs_status sedacs_graph_build_noalloc(const double* R, int32_t n_atoms, const double box[3],
                                                    double r_graph, int64_t* row_ptr, int32_t* col,
                                                    int64_t col_capacity, int64_t* nnz, void* stream) {
  if (!R || !box || !row_ptr || !col || !nnz || col_capacity < 0 || !(r_graph > 0.0)) return SEDACS_EINVAL;
  if (n_atoms <= 0 || n_atoms > kNoAllocMaxAtoms) return SEDACS_EINVAL;   // larger systems: sedacs_graph_build
  for (int a = 0; a < 3; ++a)
    if (!(box[a] > 0.0)) return SEDACS_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return SEDACS_ECUDA;
  int* scr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SEDACS_ECUDA;
      g_scratch_addr[dev] = static_cast<int*>(p);
    }
    scr = g_scratch_addr[dev];
  }
  int* counts = scr;
  int* status = scr + kNoAllocMaxAtoms;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Box3 b;
  for (int a = 0; a < 3; ++a) b.L[a] = box[a];
  const double rg2 = r_graph * r_graph;
  const int TB = 128, nb = (n_atoms + TB - 1) / TB;
  // an error left pending by the caller is not this call's: it stays for the caller to read
  if (cudaPeekAtLastError() != cudaSuccess) return SEDACS_ECUDA;
  na_count<<<nb, TB, 0, s>>>(R, n_atoms, b, rg2, counts);
  na_scan<<<1, 1024, 0, s>>>(counts, n_atoms, reinterpret_cast<long long*>(row_ptr), status, col_capacity);
  na_fill<<<nb, TB, 0, s>>>(R, n_atoms, b, rg2, reinterpret_cast<const long long*>(row_ptr), col, status);
  if (cudaGetLastError() != cudaSuccess) return SEDACS_ECUDA;    // launch errors of the three kernels
  long long total = 0;
  if (cudaMemcpyAsync(&total, row_ptr + n_atoms, sizeof(long long), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return SEDACS_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SEDACS_ECUDA;
  *nnz = total;
  return total > col_capacity ? SEDACS_ECAPACITY : SEDACS_OK;
}
