// Device kernels of the ESP long-range step and their host launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace esp {

constexpr int kMinP = 3;
constexpr int kMaxP = 12;
constexpr int kMaxDeg = 24;
// Degree of the window polynomials (Sec. 4.3, Horner): fixed per compute type so the
// coefficients of a lane's stencil point live in registers.
constexpr int kDegF32 = 13;
constexpr int kDegF64 = 24;
constexpr int kRadialPieces = 16;
constexpr int kThreads = 256;

// Geometry shared by the binning, spreading and gathering kernels.
struct TileGeom {
  int M[3];     // grid
  int P;        // stencil width
  int T[3];     // tile extent (grid points of stencil bases per tile)
  int nt[3];    // tiles per dimension
  int E[3];     // padded extent T + P - 1 of this plan's tiles (<= the TileC<P> block)
  int E3p;      // shared-memory row pitch (TileC<P>::E3p)
  int deg;      // degree of the window polynomials
  int vec4;     // 1: rows move as aligned float4 between global and shared memory
  int gvec;     // 1: the gather's block rows move as 16-byte copies (M3, T3 multiples of
                // 16 bytes of the potential grid's element type)
  int E2g;               // 16-byte pieces of a gather block row: ceil(E[2] / (16 / size))
  unsigned int div_E2g;  // ceil(2^32 / E2g)
  double hinv[9];    // h^{-1}, row-major
  float hinvf[9];    // the same in FP32 (FP32 force transform)
  double dscale[3];  // d u / d s factor of the window argument: 2 M_d / P
  float dscalef[3];
  // M_d h^{-1}[d][e] split into two floats (hi + lo) for the compensated FP32 transform
  float Ahi[9], Alo[9];
  // magic multipliers for division by E[1], by ceil(E[2] / 4) and by T[d]
  unsigned int div_E1, div_E2v, div_T[3];
  // (max |w|)^3 over the window, with a small margin: bounds |q w0 w1 w2| / |q|
  float wmax3;
};

// Constants of the fused scaling + reduction pass over the half spectrum.
struct ScaleGeom {
  int M[3];
  int H2;        // M[2]/2 + 1
  int mmax[3];   // bounding box of the sphere |k| <= K in m
  int rdeg;      // degree of the radial psi_0 / psi_0' polynomials
  double b[9];   // reciprocal vectors: k = m0 b_0 + m1 b_1 + m2 b_2, b_d = 2 pi (row d of h^{-1})
  float bf[9];
  double K2;     // (c / r_c)^2
  double x_per_k;  // r_c / c
  double A;      // 2 pi lambda_0 / C_0 = 4 pi / psi_0(0)
  double scale;  // 1 / (2 V Mtot^2)
  float K2f, x_per_kf, Af, scalef;  // FP32 copies
};

// The FFT along the first grid axis (fused with the scaling): length M0 = product of the
// pass radices (8, 4, 2, 3, 5, 7, then primes), over ncol = M1 * H2 columns taken
// 2^lognc at a time per CTA.
constexpr int kMaxPass = 32;
struct XGeom {
  int M0;
  int ncol;       // columns of the spectrum layout: nb1 * nb2
  int nb1, nb2;   // layout [M0][nb1][nb2]: the full half spectrum (M1, H2) or the box of
                  // the sphere (2 mmax1 + 1, mmax2 + 1); column (b1, m2) holds
                  // m1 = b1 for 2 b1 <= nb1, else b1 - nb1
  int lognc;
  int npass;
  int radix[kMaxPass];
  unsigned int ns_magic[kMaxPass];  // ceil(2^32 / Ns) (unused for Ns = 1), Ns = product of the radices before
};

// A mixed-radix transform of length n over nc columns held in shared memory as
// buf[j * nc + c] (j the transform index); nc is odd so that both orientations of access
// stay clear of bank conflicts.
struct LineFFT {
  int n, nc;
  int npass;
  int radix[kMaxPass];
  unsigned int ns_magic[kMaxPass];
  unsigned int nc_magic;   // ceil(2^32 / nc)
};

// The plane transforms over (i1, i2) of every plane i0, pruned to the box of the sphere
// (k_fplane forward: real grid -> box [M0][nb1][nb2]; k_iplane inverse: box -> real grid).
// Rows are taken in pairs (two real lines as one complex line), npair_b pairs per batch.
struct PlaneGeom {
  int M0, M1, M2;
  int nb1, nb2;     // the box (as XGeom)
  int mmax1;
  int npairs;       // ceil(M1 / 2)
  int pairs_b;      // pairs per batch of the transform along i2
  LineFFT a;        // along i2: n = M2, nc = pairs_b + (pairs_b even)
  LineFFT b;        // along i1: n = M1, nc = nb2 + (nb2 even)
  unsigned int m2_magic;   // ceil(2^32 / M2)
  unsigned int nb2_magic;  // ceil(2^32 / nb2)
};

struct GatherGeom {
  TileGeom g;
  double fscale;  // 1 / (V Mtot^2)
  float fscalef;  // the same in FP32 (an FP64 conversion per atom is slow on this part)
};

// Atoms binned by tile into fixed-capacity slots: the binning kernel writes atom r of
// tile t (in the order its atomics hand out) to slot t * cap + r; atoms past a tile's
// capacity go to an overflow list that spread and gather treat one atom at a time with
// global memory.  Control words (ctrl, kCtrl ints, zero between steps):
//   [0] overflow atoms of this step (binning), [1] spread tile counter, [2] spread
//   overflow counter, [3] spread CTAs done, [4] overflow atoms for the gather (set by the
//   last spread CTA), [5] gather tile counter, [6] gather overflow counter, [7] gather
//   CTAs done.  The last CTA of spread and of gather resets its own counters, and the
//   spread moves count[t] to tcount[t] and zeroes count[t].
constexpr int kCtrl = 16;
struct Bins {
  int cap;        // slots per tile
  int* count;     // [ntiles] binning counters
  int* tcount;    // [ntiles] atoms in the slots of each tile (min(count, cap))
  void* tq;       // [ntiles * cap] Vec4 of the compute type: (t0, t1, t2, q)
  int* lb;        // [ntiles * cap] stencil base relative to the tile, 10 bits per dimension
  int* idx;       // [ntiles * cap] index of the atom in the input
  void* otq;      // [n] overflow atoms (t, q)
  int* ob;        // [3 n] their stencil bases
  int* oidx;      // [n] their input indices
  int* ctrl;      // [kCtrl]
  float* hq;      // [ntiles * kHQ] FP32: sum |q| of the slotted atoms per tile and base b2
                  // (zero between steps: the spread reads and clears it)
};
constexpr int kHQ = 16;  // b2 bins per tile (T2 <= 16)

// Near (real-space) part of the split: a cell list with nc[d] >= 1 bins per reduced axis
// (each bin at least r_c / 2 thick when nc[d] > 1) and R[d] neighbour bins on either side,
// so every pair and periodic image within r_c is found exactly once.
struct NearGeom {
  int nc[3];  // cells per axis, each at least r_c / 2 wide
  int R[3];   // reach: cells per side that cover r_c
  int B[3];   // cells per block (one CTA): up to 2 x 2 x 2
  int nb[3];  // blocks per axis
  double inv_nc[3];
  double h[9];     // row-major
  double hinv[9];  // row-major
  double rc, inv_rc;
  int ndeg;        // degree of the near-kernel polynomials (kRadialPieces pieces in u)
};

// Constants of the cell gradient: h^{-1} (row-major) and U_bg = bg_coef * (sum q)^2.
struct CellGradArgs {
  double hinv[9];
  double bg_coef;
};

// Tile block of spread / gather, fixed per stencil width P so that all shared-memory
// strides are compile-time constants: a tile holds T0 x T1 x T2 stencil bases and its CTA
// owns the padded block E = T + P - 1.  Rows are padded to the pitch E3p = -P (mod 32)
// (E3p = 32 - P for these tiles) and planes to the stride S1 = P^2 (mod 32).  The point
// (i, j, k) of one atom's stencil then lies in bank (b + i P^2 + (P - 1 - j) P + k) mod 32,
// b fixed per atom: the P^3 points in the order (i, reversed j, k) fall on consecutive
// banks, so any 32 consecutive ones never share a bank.
__host__ __device__ constexpr int tile_pitch(int e2, int p) {
  int x = e2;
  while ((x + p) % 32 != 0) ++x;
  return x;
}
__host__ __device__ constexpr int plane_stride(int e1, int e3p, int p) {
  int y = e1 * e3p;
  while ((y - p * p) % 32 != 0) ++y;
  return y;
}
__host__ __device__ constexpr int round_up4(int x) { return (x + 3) & ~3; }
template <int P>
struct TileC {
  static constexpr int T0 = 8, T1 = 8, T2 = (P <= 8) ? 16 : 8;
  static constexpr int E0 = T0 + P - 1, E1 = T1 + P - 1, E2 = T2 + P - 1;
  static constexpr int E3p = tile_pitch(E2, P);
  static constexpr int S1 = plane_stride(E1, E3p, P);
  static constexpr int VOL = round_up4(E0 * S1);  // a multiple of 4 for vector clears
};
inline void tile_shape(int P, int T[3], int* E3p, int* vol) {
  T[0] = 8;
  T[1] = 8;
  T[2] = P <= 8 ? 16 : 8;
  *E3p = tile_pitch(T[2] + P - 1, P);
  *vol = round_up4((T[0] + P - 1) * plane_stride(T[1] + P - 1, *E3p, P));
}

// Atoms a CTA takes from its tile per chunk in spread / gather: all warps compute the
// window values of a chunk, then share out its atoms.
constexpr int kChunk = 128;

// Gather tile block: rows of E3 = a multiple of 16 bytes, so the block moves with 16-byte
// asynchronous copies; E3 in 16-byte units is odd, so the P rows an atom's lanes read in
// one instruction fall on distinct banks (for P <= 8 in FP32).  Two blocks (double
// buffering: the next tile's block arrives while the current one is worked on).
__host__ __device__ constexpr int gather_pitch(int e2, int es) {
  const int v = 16 / es;  // elements per 16 bytes
  int x = (e2 + v - 1) / v * v;
  if (((x / v) & 1) == 0) x += v;
  return x;
}
// atoms per chunk of the gather (its records and atom buffers)
__host__ __device__ constexpr int gather_chunk(int es) { return es == 4 ? 128 : 64; }
struct GatherLayout {
  int E3, S1, vol;           // row pitch, plane stride, block size (elements)
  size_t phi, w, tq, lb, idx, cnt, total;  // byte offsets
};
// es: compute type size; gs: size of the potential grid's element (4, 8, or 2 for BF16)
__host__ __device__ inline GatherLayout gather_layout(int es, int P, int gs) {
  GatherLayout L{};
  const int T2 = P <= 8 ? 16 : 8;
  const int E1 = 8 + P - 1, E0 = 8 + P - 1, E2 = T2 + P - 1;
  const int ch = gather_chunk(es);
  L.E3 = gather_pitch(E2, gs);
  L.S1 = E1 * L.E3;
  L.vol = E0 * L.S1;
  size_t o = 0;
  L.phi = o;  o += 2 * (size_t)L.vol * gs;                       o = (o + 31) & ~(size_t)31;
  L.w = o;    o += (size_t)ch * (6 * ((P + 3) & ~3)) * es;        o = (o + 31) & ~(size_t)31;
  L.tq = o;   o += 2 * (size_t)ch * 4 * es;                      o = (o + 31) & ~(size_t)31;
  L.lb = o;   o += 2 * (size_t)ch * sizeof(int);                 o = (o + 31) & ~(size_t)31;
  L.idx = o;  o += 2 * (size_t)ch * sizeof(int);                 o = (o + 31) & ~(size_t)31;
  L.cnt = o;  o += 2 * sizeof(int);                              o = (o + 31) & ~(size_t)31;
  L.total = o;
  return L;
}

// Per-atom record of window values in shared memory, starting on a 16-byte boundary:
// spread [w0 | q w1 | w2] (3P values, padded to a multiple of 4); gather
// [w0 | w1 | w2 | w0' | w1' | w2'], each vector in a slot of round_up4(P) values.
__host__ __device__ constexpr int record_stride(bool gather, int P) {
  return gather ? 6 * round_up4(P) : round_up4(3 * P);
}

// Spread: the padded tile block (TileC<P>, accumulators of the compute type's size), the
// chunk's window records, and two buffers of atoms ((t, q), packed local base) and counts
// for the tile worked on and the next one.
struct SpreadLayout {
  size_t w, tq, lb, cnt, hq, total;
};
__host__ __device__ inline SpreadLayout spread_layout(int es, int P) {
  SpreadLayout L{};
  int T[3] = {8, 8, P <= 8 ? 16 : 8};
  const int E3p = tile_pitch(T[2] + P - 1, P);
  const int vol = round_up4((T[0] + P - 1) * plane_stride(T[1] + P - 1, E3p, P));
  size_t o = (size_t)vol * es;
  o = (o + 31) & ~(size_t)31;
  L.w = o;   o += (size_t)kChunk * record_stride(false, P) * es;  o = (o + 31) & ~(size_t)31;
  L.tq = o;  o += 2 * (size_t)kChunk * 4 * es;                    o = (o + 31) & ~(size_t)31;
  L.lb = o;  o += 2 * (size_t)kChunk * sizeof(int);               o = (o + 31) & ~(size_t)31;
  L.cnt = o; o += 2 * sizeof(int);                                o = (o + 31) & ~(size_t)31;
  L.hq = o;  o += 2 * (size_t)kHQ * sizeof(float);                 o = (o + 31) & ~(size_t)31;
  L.total = o;
  return L;
}

// Shared-memory layout of spread / gather, byte offsets aligned to 32 bytes: the padded
// tile block, the chunk's window records, its (t, q) vectors, local bases and (gather)
// atom indices.  es = element size of the compute type (the FP32 spread accumulates 32-bit
// integers of the same size).
struct SmemLayout {
  size_t w, t, b, x, total;
};
__host__ __device__ inline size_t align32(size_t x) { return (x + 31) & ~(size_t)31; }
__host__ __device__ inline SmemLayout smem_layout(bool gather, size_t es, size_t vol, int P) {
  SmemLayout L;
  L.w = align32(vol * es);
  L.t = align32(L.w + (size_t)kChunk * record_stride(gather, P) * es);
  L.b = align32(L.t + (size_t)kChunk * 4 * es);
  L.x = align32(L.b + (size_t)kChunk * sizeof(int));
  L.total = align32(L.x + (gather ? (size_t)kChunk * sizeof(int) : 0));
  return L;
}

// ---- launchers (return cudaGetLastError() of the launch) -----------------------------
// io_double: pos/q/F are double (else float).  fp64: compute type double (else float).

// Wrap, stencil base and slot of every atom (Bins); also clears zero_bytes of zero_buf
// (the spread target grid), by a memset when n <= 0.  bin_part: per block 3 compensated
// sums (sum q, sum q^2, skipped atoms) as float pairs.
cudaError_t launch_bin(bool io_double, bool fp64, const void* pos, const void* q, int64_t n,
                       const TileGeom& g, const Bins& b, void* bin_part, void* zero_buf,
                       size_t zero_bytes, cudaStream_t st);
int bin_blocks(int64_t n);
// slots per tile for n atoms over ntiles tiles (about 2.5x the mean, at least 32)
int bin_capacity(int64_t n, int ntiles);
cudaError_t launch_spread(bool fp64, const TileGeom& g, int ntiles, int nblocks, const Bins& b,
                          const void* wtab, void* grid, cudaStream_t st);
// The transform along axis 0 fused with the scaling (k_xfft, kXThreads per CTA): the
// sums of U_F and W_F over the sphere; fwd: the columns first take the forward transform
// along axis 0 (the planes are transformed), else they hold the full 3D spectrum; inv: the
// scaled modes take the inverse transform along axis 0 and go to out, of which only the
// active columns are written (the caller clears out first); fwd needs inv.  tw: M0 roots e^{-2 pi i m / M0}
// of the compute type.  order: the xfft_blocks(x) column groups, the nactive (>= 1)
// groups holding every column with colact[f] = 1 first.  colact: per column, 1 if its line
// k = m0 b_0 + m1 b_1 + m2 b_2 may enter the sphere |k| <= K.  partials: 7 x nactive
// doubles (per-CTA sums of U_F and W_F xx yy zz xy xz yz); launch_xsum(partials, nactive)
// adds them into accum[0..6], and the binning partials (bin_part: per binning block 3
// compensated sums as float pairs; nbin blocks, 0 for no atoms) into accum[7..9].
constexpr int kXThreads = 512;
int xfft_blocks(const XGeom& x);
size_t xfft_smem_bytes(bool fp64, int M0, int lognc, int rdeg);
cudaError_t configure_xfft(bool fp64, size_t smem);
cudaError_t launch_xfft(bool fp64, bool fwd, bool inv, const XGeom& x, const ScaleGeom& s,
                        const void* spec, void* out, const void* tw, const void* invw2,
                        const void* radtab,
                        double* partials, const int* order, const unsigned char* colact,
                        int nactive, cudaStream_t st);
// nf floats src -> dst (dst: the device mapping of page-locked host memory; both 16-byte
// aligned) and nacc doubles acc -> acc_dst, on 2 sms CTAs.
cudaError_t launch_copy_out(const void* src, void* dst, int64_t nf, const double* acc,
                            double* acc_dst, int nacc, int sms, cudaStream_t st);
cudaError_t launch_xsum(bool fp64, const double* partials, int nblk, const void* bin_part,
                        int nbin, double* accum, cudaStream_t st);
// Plane transforms (2 kPThreads per CTA in FP32, kPThreads in FP64; one CTA per plane i0).  tw: M1 roots
// e^{-2 pi i m / M1} then M2 roots e^{-2 pi i m / M2} of the compute type.  fplane: grid
// (M0 x M1 x M2 real) -> box (M0 x nb1 x nb2 complex).  iplane: box -> grid, columns with
// colact = 0 read as zero (k_xfft writes only the active ones).
constexpr int kPThreads = 512;
size_t plane_smem_bytes(bool fp64, const PlaneGeom& pg);
cudaError_t configure_planes(bool fp64, size_t smem);
cudaError_t launch_fplane(bool fp64, const PlaneGeom& pg, const void* grid, void* box,
                          const void* tw, cudaStream_t st);
cudaError_t launch_iplane(bool fp64, bool bf16, const PlaneGeom& pg, const void* box,
                          const unsigned char* colact, void* grid, const void* tw,
                          cudaStream_t st);
// bf16: the potential grid is BF16 (FP32 compute only)
cudaError_t launch_gather(bool fp64, bool io_double, bool bf16, const GatherGeom& gg, int ntiles,
                          int nblocks, const Bins& b, const void* wtab, const void* grid,
                          void* forces, cudaStream_t st);
// Near part.  bin: cell id, rank within the cell and the atom's position relative to its
// cell corner (with q) in the input order; ccount (ncells ints) zero on entry.  scan:
// coff[0..ncells] exclusive offsets, ccount zeroed again.  scatter: cell order, and
// xq_tmp zeroed (it is the pairs' sorted-order force accumulator fsort).  pairs: half-shell
// pair sums over blocks of B cells, then the forces to the caller's array in input order
// (overwritten, or added to when add != 0), out[0..6] = U_N, W_N xx yy zz xy xz yz
// (overwritten).
constexpr int kNearMaxRegion = 2048;  // cells of one block's neighbourhood
constexpr int kNearMaxHome = 8;       // cells of one block (at most 2 x 2 x 2)
constexpr size_t kNearMaxSmem = 200 * 1024;  // dynamic shared memory of the pair kernel
int near_region_cells(const NearGeom& ng);
size_t near_pairs_smem(bool fp64, const NearGeom& ng);
cudaError_t launch_near_bin(bool io_double, bool fp64, const void* pos, const void* q,
                            int64_t n, const NearGeom& ng, int* ccount, int* cell, int* rank,
                            void* xq_tmp, cudaStream_t st);
cudaError_t launch_near_scan(int* ccount, int* coff, int ncells, cudaStream_t st);
cudaError_t launch_near_scatter(bool fp64, int64_t n, const int* cell, const int* rank,
                                const int* coff, void* xq_tmp, void* xq, int* idx,
                                cudaStream_t st);
// offtab: kNearMaxRegion vec4 of the compute type (device scratch, written here)
cudaError_t launch_near_pairs(bool fp64, bool io_double, const NearGeom& ng, int ncells,
                              const int* coff, const void* xq, const int* idx, const void* tab,
                              void* offtab, void* fsort, void* forces, int add, int64_t n,
                              double* out, cudaStream_t st);

// Fields from the kept spectrum (kind 0: G X; 1: i k_d G X; 2: K_ab X / w^2), written as
// 1, 3 or 6 half spectra one after the other.
cudaError_t launch_fields(bool fp64, int kind, const ScaleGeom& s, const void* spec,
                          const void* invw2, const void* radtab, void* out, cudaStream_t st);
// Window interpolation of nf (1 or 3) real grids at the atoms (grids field_stride apart):
// out[idx * stride + off + f] = coef q_i sum_g field_f(g) w(g / M - s_i); uses the gather's
// control words.
cudaError_t launch_gather_fields(bool fp64, bool io_double, const TileGeom& g, int ntiles,
                                 int nblocks, int nf, const Bins& b, const void* wtab,
                                 const void* fields, int64_t field_stride, double coef,
                                 void* out, int stride, int off, cudaStream_t st);
size_t fields_smem_bytes(bool fp64, int P, int NF);

// dU/dh at fixed positions into grad[9] (row-major): -W h^{-T} + sum_i F_i (h^{-1} r_i)^T
cudaError_t launch_cell_grad(bool io_double, const void* pos, const void* forces, int64_t n,
                             const CellGradArgs& c, const double* accum, double* grad,
                             cudaStream_t st);
cudaError_t occupancy(bool fp64, bool io_double, int P, size_t spread_smem, size_t gather_smem,
                      int* spread_ctas, int* gather_ctas, bool bf16 = false);

size_t spread_smem_bytes(bool fp64, const TileGeom& g);
size_t gather_smem_bytes(bool fp64, const TileGeom& g, bool bf16 = false);
cudaError_t configure_kernels(bool fp64, int P, size_t spread_smem, size_t gather_smem,
                              bool bf16 = false);

}  // namespace esp
