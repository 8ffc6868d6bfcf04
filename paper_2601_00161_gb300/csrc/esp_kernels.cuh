// Device kernels of the ESP long-range step and their host launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace esp {

constexpr int kMinP = 3;
constexpr int kMaxP = 12;
constexpr int kMaxDeg = 24;
constexpr int kRadialPieces = 16;
constexpr int kThreads = 256;

// Geometry shared by the binning, spreading and gathering kernels.
struct TileGeom {
  int M[3];     // grid
  int P;        // stencil width
  int T[3];     // tile extent (grid points of stencil bases per tile)
  int nt[3];    // tiles per dimension
  int E[3];     // padded tile extent T + P - 1
  int E3p;      // padded row pitch in shared memory (>= E[2])
  int deg;      // degree of the window polynomials
  double hinv[9];  // h^{-1}, row-major
};

// Constants of the fused scaling + reduction pass over the half spectrum.
struct ScaleGeom {
  int M[3];
  int H2;        // M[2]/2 + 1
  int mmax[3];   // bounding box of the sphere |k| <= K in m
  int rdeg;      // degree of the radial psi_0 / psi_0' polynomials
  double b[9];   // reciprocal vectors: k = m0 b_0 + m1 b_1 + m2 b_2, b_d = 2 pi (row d of h^{-1})
  double K2;     // (c / r_c)^2
  double x_per_k;  // r_c / c
  double A;      // 2 pi lambda_0 / C_0 = 4 pi / psi_0(0)
  double scale;  // 1 / (2 V Mtot^2)
};

struct GatherGeom {
  TileGeom g;
  double fscale;  // 1 / (V Mtot^2)
};

// ---- launchers (return cudaGetLastError() of the launch) -----------------------------
// io_double: pos/q/F are double (else float).  R: compute type via `fp64`.

cudaError_t launch_bin(bool io_double, const void* pos, const void* q, int64_t n,
                       const TileGeom& g, int* tile_count, int* ptile, int* prank, int* plb,
                       double* accum, cudaStream_t st);
cudaError_t launch_scan(const int* count, int* offset, int ntiles, cudaStream_t st);
cudaError_t launch_scatter(bool io_double, bool fp64, const void* pos, const void* q,
                           int64_t n, const TileGeom& g, const int* ptile, const int* prank,
                           const int* plb, const int* offset, void* sorted_tq, int* sorted_lb, int* sorted_idx,
                           cudaStream_t st);
cudaError_t launch_spread(bool fp64, const TileGeom& g, int ntiles, const void* sorted_tq,
                          const int* sorted_lb, const int* offset, const void* wtab,
                          void* grid, cudaStream_t st);
cudaError_t launch_scale(bool fp64, bool write, const ScaleGeom& s, void* spec,
                         const void* invw2, const void* radtab, double* partials,
                         unsigned int* counter, double* accum, int nblocks, cudaStream_t st);
cudaError_t launch_gather(bool fp64, bool io_double, const GatherGeom& gg, int ntiles,
                          const void* sorted_tq, const int* sorted_lb, const int* sorted_idx,
                          const int* offset, const void* wtab, const void* grid, void* forces,
                          cudaStream_t st);

size_t spread_smem_bytes(bool fp64, const TileGeom& g);
size_t gather_smem_bytes(bool fp64, const TileGeom& g);
cudaError_t configure_kernels(bool fp64, int P, size_t spread_smem, size_t gather_smem);

}  // namespace esp
