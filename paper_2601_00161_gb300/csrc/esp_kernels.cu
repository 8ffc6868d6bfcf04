// sm_103a kernels of the ESP long-range step (Sec. 4.1 Algorithm 1 and Appendix C):
//   k_bin      wrap s = h^{-1} r into [0,1), stencil base and fractional offset
//              (Sec. 4.3), tile id; the atom goes straight to the next free slot of its
//              tile (warp-aggregated atomics; past the tile's capacity, to an overflow
//              list); the integer stencil decision is taken in FP64 near a switch so it
//              matches the FP64 oracle
//   k_spread   eq. (gridding): persistent CTAs stage a tile's padded block in shared
//              memory; a warp adds one atom's P^3 footprint at a time along lane-fixed
//              stencil columns (32 distinct banks per add), as 32-bit fixed point with
//              the native shared-memory integer add and a per-tile scale from the binned
//              charge sums; the block then goes to the periodic grid with vector
//              reductions
//   k_fplane   the plane transforms over (i1, i2) of one plane i0 per CTA, pruned to the
//              box of the sphere (two real lines as one complex line along i2, then the
//              kept columns along i1)
//   k_xfft     the transform along the first grid axis of the column groups whose lines
//              meet the sphere |k| <= c / r_c (mixed-radix Stockham passes in shared
//              memory), fused with eqs. (diag)/(PFfinal): per mode the deconvolved weight,
//              the Fourier kernel and the 3x3 pressure kernel, summed per CTA (compensated
//              FP32 on the FP32 path), and for forces G X and the inverse transform
//   k_xsum     the fixed-order final sums of k_xfft's partials and of the charge sums
//   k_iplane   the inverse of k_fplane from the scaled box into the potential grid
//   k_gather   eq. (AD): the CTA stages its tile's padded block of the potential grid in
//              shared memory; P lanes per atom contract its P^3 points with the window
//              and its gradient, a segmented shuffle sums them
// Around the step: k_cell_grad (cell gradient, Sec. 2.2), k_fields and k_gather_fields
// (ik forces, local virial, per-atom energy: Sec. 4.4, Appendix C), the near part of the
// split (k_near_bin, k_near_scan, k_near_scatter, k_near_offsets, k_near_pairs,
// k_near_out: Sec. 3, eq. (UN)) and k_copy_out (results to page-locked host memory).
//
// Shared-memory layout of a tile block: row pitch E3p = -P (mod 32) and plane stride
// S1 = P^2 (mod 32), so the stencil point (i, j, k) of an atom lies in bank
// (b + i P^2 + (P - 1 - j) P + k) mod 32 and 32 consecutive points in the order
// (i, reversed j, k) never share a bank.
#include "esp_kernels.cuh"

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <utility>

namespace esp {

namespace {

template <typename R>
struct Vec4;
template <>
struct Vec4<float> {
  using T = float4;
};
template <>
struct Vec4<double> {
  using T = double4;
};

template <typename R>
struct Cplx;
template <>
struct Cplx<float> {
  using T = float2;
};
template <>
struct Cplx<double> {
  using T = double2;
};

// Elements of the potential grid: the compute type, or BF16 (read into FP32).
__device__ __forceinline__ float grid_val(float x) { return x; }
__device__ __forceinline__ double grid_val(double x) { return x; }
__device__ __forceinline__ float grid_val(__nv_bfloat16 x) { return __bfloat162float(x); }
template <typename G, typename R>
__device__ __forceinline__ G grid_elem(R x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 grid_elem<__nv_bfloat16, float>(float x) {
  return __float2bfloat16_rn(x);
}

__device__ __forceinline__ int wrap_index(int i, int m) {
  i %= m;
  return i < 0 ? i + m : i;
}

// floor(x / d) for 0 <= x < 2^16 with m = ceil(2^32 / d), d < 2^16
__device__ __forceinline__ int fast_div(int x, unsigned int m) {
  return (int)__umulhi((unsigned int)x, m);
}

// x in [0, 3 m) -> x mod m
// Programmatic dependent launch: a kernel launched with programmatic stream serialization
// may start while the kernel before it finishes; it waits here before touching that
// kernel's results (a no-op for a plain launch).  The trigger lets the next kernel's CTAs
// be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }

// Asynchronous copies global -> shared (cp.async; no register staging).  16 bytes need
// 16-byte aligned addresses on both sides.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ int wrap3(int x, int m) {
  x = x >= m ? x - m : x;
  return x >= m ? x - m : x;
}

// Compensated ("double-float") FP32 arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
struct DF {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float v) {
    float s, e;
    two_sum(hi, v, s, e);
    hi = s;
    lo += e;
  }
  __device__ __forceinline__ void add(const DF& o) {
    float s, e;
    two_sum(hi, o.hi, s, e);
    hi = s;
    lo += o.lo + e;
  }
};

// Reduced coordinate, grid coordinate and stencil base for one dimension (Sec. 4.3):
// P even: base = floor(x) - P/2 + 1, t = x - floor(x); P odd: base = floor(x + 1/2) -
// (P-1)/2, t = x + 1/2 - floor(x + 1/2).  Either way stencil point p sits at offset
// g - x = p + 1 - P/2 - t from the atom, in grid units.  Explicitly rounded FP64.
__device__ __forceinline__ void stencil_base(double s, int M, int P, int* base, double* t) {
  s = __dsub_rn(s, floor(s));
  if (s >= 1.0) s = 0.0;
  double x = __dmul_rn((double)M, s);
  if (P & 1) x = __dadd_rn(x, 0.5);
  const double fl = floor(x);
  *t = __dsub_rn(x, fl);
  int b = (int)fl - ((P & 1) ? (P - 1) / 2 : P / 2 - 1);  // in [-P/2, M]
  b = b < 0 ? b + M : (b >= M ? b - M : b);
  *base = b;
}

__device__ __forceinline__ double reduced_coord(const double* hinv_row, const double r[3]) {
  return __fma_rn(hinv_row[0], r[0], __fma_rn(hinv_row[1], r[1], __dmul_rn(hinv_row[2], r[2])));
}

// The grid coordinate x = M_d (h^{-1} r)_d of FP32 positions in compensated FP32: exact
// products (FMA) of the float pair A = M_d h^{-1}[d][.] with r, compensated sums.  Its
// error is ~|x| 2^-46, so the integer part agrees with the FP64 computation except when
// x lies within that distance of an integer; any x within 1e-6 of an integer (or too
// large for the float pair) returns false and the caller takes the FP64 decision.
__device__ __forceinline__ bool stencil_base_df(const TileGeom& g, int d, const float* r,
                                                int* base, float* t_out) {
  float S = 0.f, err = 0.f;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const float hi = g.Ahi[3 * d + e];
    const float p = hi * r[e];
    const float pe = fmaf(hi, r[e], -p);  // exact: hi * r = p + pe
    float s2, e2;
    two_sum(S, p, s2, e2);
    S = s2;
    err += e2 + pe + g.Alo[3 * d + e] * r[e];
  }
  if (g.P & 1) {
    float s2, e2;
    two_sum(S, 0.5f, s2, e2);
    S = s2;
    err += e2;
  }
  if (!(fabsf(S) < 1048576.f)) return false;
  float fl = floorf(S);
  float t = (S - fl) + err;  // S - fl is exact
  if (t < 0.f) {
    t += 1.f;
    fl -= 1.f;
  } else if (t >= 1.f) {
    t -= 1.f;
    fl += 1.f;
  }
  if (t < 1e-6f || t > 1.f - 1e-6f) return false;
  const int M = g.M[d];
  int b = (int)fl - ((g.P & 1) ? (g.P - 1) / 2 : g.P / 2 - 1);
  if ((unsigned)b >= (unsigned)M) {  // an atom outside the primary cell (rare): wrap
    b %= M;
    if (b < 0) b += M;
  }
  *base = b;
  *t_out = t;
  return true;
}


__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename R>
__device__ __forceinline__ R dscale_of(const TileGeom& g, int d);
template <>
__device__ __forceinline__ float dscale_of<float>(const TileGeom& g, int d) {
  return g.dscalef[d];
}
template <>
__device__ __forceinline__ double dscale_of<double>(const TileGeom& g, int d) {
  return g.dscale[d];
}

// ---------------------------------------------------------------------------------------
template <typename IO, typename R>
__global__ void __launch_bounds__(kThreads, 6) k_bin(const IO* __restrict__ pos,
                                                  const IO* __restrict__ q, int64_t n,
                                                  TileGeom g, Bins bins,
                                                  float2* __restrict__ bin_part,
                                                  int4* __restrict__ zero, int64_t nzero) {
  pdl_trigger();
  using V4 = typename Vec4<R>::T;
  // FP32 inputs on the FP32 path use the compensated FP32 transform (FP64 only for the
  // rare coordinate next to a stencil switch); everything else uses FP64.
  constexpr bool kDF = std::is_same<IO, float>::value && std::is_same<R, float>::value;
  // the spread target grid is cleared here too (nzero 16-byte words), saving a memset
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nzero;
       i += (int64_t)gridDim.x * blockDim.x)
    zero[i] = make_int4(0, 0, 0, 0);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lanes_below = (1u << lane) - 1u;
  V4* slot_tq = static_cast<V4*>(bins.tq);
  DF sq, sq2, bad;
  // uniform trip count per warp: the slot ranks are handed out per warp
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < n; i0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = i0 + threadIdx.x;
    int tile = -1, lbp = 0, b[3] = {0, 0, 0};
    V4 v{};
    if (i < n) {
      const IO r0 = pos[3 * i], r1 = pos[3 * i + 1], r2 = pos[3 * i + 2], qi = q[i];
      if (!(isfinite(r0) && isfinite(r1) && isfinite(r2) && isfinite(qi))) {
        bad.add(1.f);
      } else {
        int tc[3], lb[3];
        R t[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          bool done = false;
          if constexpr (kDF) {
            const float rf[3] = {(float)r0, (float)r1, (float)r2};
            done = stencil_base_df(g, d, rf, &b[d], &t[d]);
          }
          if (!done) {
            const double r[3] = {(double)r0, (double)r1, (double)r2};
            double td;
            stencil_base(reduced_coord(&g.hinv[3 * d], r), g.M[d], g.P, &b[d], &td);
            t[d] = (R)td;
          }
          tc[d] = fast_div(b[d], g.div_T[d]);  // b < 4096, T <= 16
          lb[d] = b[d] - tc[d] * g.T[d];
        }
        tile = (tc[0] * g.nt[1] + tc[1]) * g.nt[2] + tc[2];
        v.x = t[0];
        v.y = t[1];
        v.z = t[2];
        v.w = (R)qi;
        lbp = lb[0] | (lb[1] << 10) | (lb[2] << 20);
        if constexpr (std::is_same<IO, float>::value) {
          sq.add(qi);
          sq2.add(qi * qi);
        } else {
          // split the double into a float pair so the sums stay accurate to ~2^-48
          const float qh = (float)qi, ql = (float)(qi - (double)qh);
          const double q2 = qi * qi;
          const float q2h = (float)q2, q2l = (float)(q2 - (double)q2h);
          sq.add(qh);
          sq.add(ql);
          sq2.add(q2h);
          sq2.add(q2l);
        }
      }
    }
    // lanes of one tile take consecutive slots with one atomic per tile and warp
    const unsigned same = __match_any_sync(0xffffffffu, tile);
    const int leader = __ffs(same) - 1;
    int first = 0;
    if (lane == leader && tile >= 0) first = atomicAdd(&bins.count[tile], __popc(same));
    first = __shfl_sync(0xffffffffu, first, leader);
    if (tile >= 0) {
      const int r = first + __popc(same & lanes_below);
      if (r < bins.cap) {
        const int64_t sl = (int64_t)tile * bins.cap + r;
        slot_tq[sl] = v;
        bins.lb[sl] = lbp;
        bins.idx[sl] = (int)i;
        // the FP32 spread's fixed-point bound: sum |q| per tile and base b2
        if constexpr (std::is_same<R, float>::value)
          atomicAdd(bins.hq + (int64_t)tile * kHQ + (lbp >> 20), fabsf(v.w));
      } else {
        const int o = atomicAdd(&bins.ctrl[0], 1);
        static_cast<V4*>(bins.otq)[o] = v;
        bins.ob[3 * o] = b[0];
        bins.ob[3 * o + 1] = b[1];
        bins.ob[3 * o + 2] = b[2];
        bins.oidx[o] = (int)i;
      }
    }
  }
  // compensated warp sums, then one compensated pair per block (k_xsum adds them up)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF a, b2, c;
    a.hi = __shfl_xor_sync(0xffffffffu, sq.hi, o);
    a.lo = __shfl_xor_sync(0xffffffffu, sq.lo, o);
    b2.hi = __shfl_xor_sync(0xffffffffu, sq2.hi, o);
    b2.lo = __shfl_xor_sync(0xffffffffu, sq2.lo, o);
    c.hi = __shfl_xor_sync(0xffffffffu, bad.hi, o);
    c.lo = __shfl_xor_sync(0xffffffffu, bad.lo, o);
    sq.add(a);
    sq2.add(b2);
    bad.add(c);
  }
  __shared__ float2 red[3][kThreads / 32];
  if (lane == 0) {
    red[0][wid] = make_float2(sq.hi, sq.lo);
    red[1][wid] = make_float2(sq2.hi, sq2.lo);
    red[2][wid] = make_float2(bad.hi, bad.lo);
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    DF a;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      DF y;
      y.hi = red[threadIdx.x][w].x;
      y.lo = red[threadIdx.x][w].y;
      a.add(y);
    }
    bin_part[3 * blockIdx.x + threadIdx.x] = make_float2(a.hi, a.lo);
  }
}

// The CTA that finishes last resets the control words [first, first + cnt) of its kernel
// (counters zero again for the next step).  Every CTA must reach this point.
__device__ __forceinline__ void last_cta_resets(int* ctrl, int done_word, int first, int cnt,
                                                int copy_from = -1, int copy_to = -1) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const int done = atomicAdd(&ctrl[done_word], 1);
    if (done == (int)gridDim.x - 1) {
      __threadfence();
      volatile int* vc = ctrl;
      if (copy_from >= 0) {
        vc[copy_to] = vc[copy_from];
        vc[copy_from] = 0;
      }
      for (int k = 0; k < cnt; ++k) vc[first + k] = 0;
      __threadfence();
    }
  }
}

template <typename R>
struct WinDeg;
template <>
struct WinDeg<float> {
  static constexpr int value = kDegF32;
};
template <>
struct WinDeg<double> {
  static constexpr int value = kDegF64;
};

// Vector reduction of four floats into global memory (no value returned, so no register
// waits for the atomic to complete).  addr: 16-byte aligned.
__device__ __forceinline__ void red_add4(void* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
               "f"(c), "f"(d)
               : "memory");
}

// Horner with the coefficients of (t - 1/2)^k held in registers
template <typename R, int D>
__device__ __forceinline__ R horner_reg(const R (&c)[D + 1], R t) {
  const R tau = t - R(0.5);
  R v = c[D];
#pragma unroll
  for (int k = D - 1; k >= 0; --k) v = fma(v, tau, c[k]);
  return v;
}

// Two FP32 Horner evaluations in step, as packed pairs (fma.rn.f32x2: each half rounds as
// a separate fma.rn, so the values equal those of two horner_reg calls).
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2(unsigned long long r, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
// tau holds the packed argument t - 1/2 of both polynomials
template <int D>
__device__ __forceinline__ unsigned long long horner2(const unsigned long long (&c)[D + 1],
                                                      unsigned long long tau) {
  unsigned long long v = c[D];
#pragma unroll
  for (int k = D - 1; k >= 0; --k) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(v) : "l"(tau), "l"(c[k]));
  return v;
}

template <typename R>
__device__ __forceinline__ R tq_comp(const typename Vec4<R>::T& v, int d) {
  return d == 0 ? v.x : (d == 1 ? v.y : v.z);
}


// offset of an atom's stencil corner in the padded tile block (packed local base: 10 bits
// per dimension)
template <int S1, int E3p>
__device__ __forceinline__ int local_base(int lb) {
  return (lb & 1023) * S1 + ((lb >> 10) & 1023) * E3p + ((lb >> 20) & 1023);
}

// P values of a 16-byte aligned shared-memory record into registers (vector loads)
template <typename R, int P>
__device__ __forceinline__ void load_record(const R* src, R (&dst)[P]) {
  if constexpr (std::is_same<R, float>::value) {
#pragma unroll
    for (int i = 0; i + 4 <= P; i += 4) {
      const float4 v = *reinterpret_cast<const float4*>(src + i);
      dst[i] = v.x;
      dst[i + 1] = v.y;
      dst[i + 2] = v.z;
      dst[i + 3] = v.w;
    }
    constexpr int r = P & ~3;
    if constexpr (P - r >= 2) {
      const float2 v = *reinterpret_cast<const float2*>(src + r);
      dst[r] = v.x;
      dst[r + 1] = v.y;
    }
    if constexpr ((P - r) & 1) dst[P - 1] = src[P - 1];
  } else {
#pragma unroll
    for (int i = 0; i + 2 <= P; i += 2) {
      const double2 v = *reinterpret_cast<const double2*>(src + i);
      dst[i] = v.x;
      dst[i + 1] = v.y;
    }
    if constexpr (P & 1) dst[P - 1] = src[P - 1];
  }
}

// Lane-fixed stencil columns.  A warp works on one atom at a time.  A column is a pair
// (j, k) numbered c = (P - 1 - j) P + k; in full pass m lane l owns column c = 32 m + l and
// walks i = 0 .. P-1, and for each i the 32 lanes touch 32 consecutive banks (see TileC).
// The NT = P^2 mod 32 leftover columns give NT P tail points, handed out 32 at a time in
// the order u = i NT + (c - 32 MP), whose banks are again consecutive.
template <int P>
struct Cols {
  static constexpr int MP = P * P / 32;
  static constexpr int NT = P * P % 32;
  static constexpr int NG = (NT * P + 31) / 32;
};

// Per-lane tables of the columns: full passes (offset in the block, j and k) and tail points
// packed as offset | i << 16 | j << 20 | k << 24 | valid << 31.
template <int P, int S1, int E3p>
struct LaneCols {
  int off[Cols<P>::MP > 0 ? Cols<P>::MP : 1];
  int j[Cols<P>::MP > 0 ? Cols<P>::MP : 1];
  int k[Cols<P>::MP > 0 ? Cols<P>::MP : 1];
  unsigned tail[Cols<P>::NG > 0 ? Cols<P>::NG : 1];
  // the same tail points unpacked for the spread: byte offset of a 4- or 8-byte element,
  // record indices of w0[i], q w1[j] and w2[k], and whether the lane has a point
  int tail_off[Cols<P>::NG > 0 ? Cols<P>::NG : 1];
  int tail_i[Cols<P>::NG > 0 ? Cols<P>::NG : 1], tail_j[Cols<P>::NG > 0 ? Cols<P>::NG : 1],
      tail_k[Cols<P>::NG > 0 ? Cols<P>::NG : 1];
  bool tail_ok[Cols<P>::NG > 0 ? Cols<P>::NG : 1];
  __device__ __forceinline__ LaneCols(int lane, int elem_bytes) : LaneCols(lane) {
#pragma unroll
    for (int g = 0; g < (Cols<P>::NG > 0 ? Cols<P>::NG : 1); ++g) {
      const unsigned tp = tail[g];
      tail_ok[g] = (tp >> 31) != 0u;
      tail_off[g] = (int)(tp & 0xffffu) * elem_bytes;
      tail_i[g] = (tp >> 16) & 15;
      tail_j[g] = P + ((tp >> 20) & 15);
      tail_k[g] = 2 * P + ((tp >> 24) & 15);
    }
  }
  __device__ __forceinline__ explicit LaneCols(int lane) {
    using C = Cols<P>;
#pragma unroll
    for (int m = 0; m < C::MP; ++m) {
      const int c = 32 * m + lane;
      j[m] = P - 1 - c / P;
      k[m] = c - (c / P) * P;
      off[m] = j[m] * E3p + k[m];
    }
    tail[0] = 0u;
    if constexpr (C::NT > 0) {
#pragma unroll
      for (int g = 0; g < C::NG; ++g) {
        const int u = 32 * g + lane;
        tail[g] = 0u;
        if (u < C::NT * P) {
          const int i = u / C::NT;
          const int c = 32 * C::MP + (u - i * C::NT);
          const int jj = P - 1 - c / P, kk = c - (c / P) * P;
          tail[g] = (unsigned)(i * S1 + jj * E3p + kk) | ((unsigned)i << 16) |
                    ((unsigned)jj << 20) | ((unsigned)kk << 24) | (1u << 31);
        }
      }
    }
  }
};

// Accumulation into the spread block: FP32 values as 32-bit fixed point (value x scale,
// rounded to nearest) with the native shared-memory integer add, FP64 values with the
// double atomic add.  OFF is a compile-time byte offset from the shared-space address.
template <int OFF>
__device__ __forceinline__ void red_fixed(unsigned addr, float v) {
  asm volatile("red.shared.add.s32 [%0+%2], %1;" ::"r"(addr), "r"(__float2int_rn(v)), "n"(OFF)
               : "memory");
}
template <int OFF>
__device__ __forceinline__ void red_fixed(unsigned addr, double v) {
  atomicAdd(reinterpret_cast<double*>(__cvta_shared_to_generic(addr + OFF)), v);
}
// one column of an atom: the P values w0[i] * pw at the offsets i * S1 from the column start
template <typename R, int S1, int... I>
__device__ __forceinline__ void spread_column(unsigned addr, const R (&w0)[sizeof...(I)], R pw,
                                              std::integer_sequence<int, I...>) {
  (red_fixed<I * S1 * (int)sizeof(R)>(addr, w0[I] * pw), ...);
}
// FP32: the same with the products taken as packed pairs (mul.rn.f32x2 rounds each half
// as mul.rn): w0p[m] holds (w0[2m], w0[2m + 1]), pw2 holds (pw, pw)
template <int S1, int P, int... M>
__device__ __forceinline__ void spread_column2(unsigned addr,
                                               const unsigned long long (&w0p)[(P + 1) / 2],
                                               unsigned long long pw2,
                                               std::integer_sequence<int, M...>) {
  auto one = [&](auto mc) {
    constexpr int m = decltype(mc)::value;
    unsigned long long pr;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(pr) : "l"(w0p[m]), "l"(pw2));
    float lo, hi;
    unpack2(pr, lo, hi);
    red_fixed<2 * m * S1 * 4>(addr, lo);
    if constexpr (2 * m + 1 < P) red_fixed<(2 * m + 1) * S1 * 4>(addr, hi);
  };
  (one(std::integral_constant<int, M>{}), ...);
}

// ---------------------------------------------------------------------------------------
// Five resident CTAs per SM where 48 registers hold the FP32 spread without spills.
template <typename R, int P>
constexpr int spread_min_ctas() {
  return (std::is_same<R, float>::value && (P == 3 || P == 4 || P == 6 || P == 8)) ? 5 : 1;
}

// Persistent CTAs take tiles from a global counter (ctrl[1]) two ahead of the one they
// work on; the next tile's atom count and first chunk of atoms arrive by asynchronous
// copies into the other half of a double buffer while the current tile is worked on.
// Per chunk of a tile's atoms: (A) thread (p, a) evaluates the window at stencil point p
// for the three dimensions of atom a (coefficients in registers); (B) each warp takes one
// atom at a time and adds its P^3 values into the padded block along the lane-fixed
// columns of Cols<P>, every shared-memory add of the warp hitting 32 distinct banks.  The
// FP32 block holds 32-bit fixed point with a power-of-two scale per tile: scale <= 2^30 /
// (max |w|^3 x the largest sum of |q| over the atoms whose bases fall in a window of P
// positions along axis 2), so no partial sum can overflow; the rounding of each
// contribution is at most half a unit of 2^-30 times that bound.  The block then goes to
// the periodic grid with global vector reductions, and is cleared as it is read.
template <typename R, int P>
__global__ void __launch_bounds__(kThreads, spread_min_ctas<R, P>()) k_spread(Bins bins, TileGeom g, int ntiles,
                                                     const R* __restrict__ wtab,
                                                     R* __restrict__ grid) {
  pdl_wait();
  using V4 = typename Vec4<R>::T;
  const V4* __restrict__ slot_tq = static_cast<const V4*>(bins.tq);
  using TC = TileC<P>;
  using CM = Cols<P>;
  constexpr bool kFixed = std::is_same<R, float>::value;
  using A = typename std::conditional<kFixed, int, double>::type;  // accumulator element
  extern __shared__ __align__(16) unsigned char smem_raw[];
  A* acc = reinterpret_cast<A*>(smem_raw);
  constexpr int E1 = TC::E1, E3p = TC::E3p, vol = TC::VOL, S1 = TC::S1;
  constexpr int RS = record_stride(false, P);
  const int E0 = g.E[0], E2 = g.E[2];  // this plan's tiles (<= TC)
  const SpreadLayout L = spread_layout((int)sizeof(R), P);
  R* W = reinterpret_cast<R*>(smem_raw + L.w);        // per atom [w0 | q w1 | w2]
  float* HQ_b = reinterpret_cast<float*>(smem_raw + L.hq);  // 2 x kHQ: the tile's sum |q| per b2
  V4* TQ_b = reinterpret_cast<V4*>(smem_raw + L.tq);  // 2 x kChunk (t0, t1, t2, q)
  int* LB_b = reinterpret_cast<int*>(smem_raw + L.lb);
  int* CNT_b = reinterpret_cast<int*>(smem_raw + L.cnt);
  // tiles taken ahead, with the grid origin of each (computed once, by the thread that
  // takes the tile)
  __shared__ int s_first[2], s_ahead[2];
  __shared__ int3 s_ofirst[2], s_oahead[2];
  __shared__ float s_bound;  // FP32: the tile's bound of sum |q|
  const unsigned acc_s = (unsigned)__cvta_generic_to_shared(acc);

  constexpr int D = WinDeg<R>::value;
  constexpr int NPA = kThreads / P;  // atoms per sweep of the window evaluation
  const int p_t = threadIdx.x % P, a_t = threadIdx.x / P;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const LaneCols<P, S1, E3p> lc(lane, (int)sizeof(A));
  const int ncopy = min(kChunk, bins.cap);

  // copies of tile t into buffer b: its binning count and first chunk of atoms
  auto issue = [&](int t, int b) {
    if (t < ntiles) {
      const int64_t s0 = (int64_t)t * bins.cap;
      constexpr int QV = (int)sizeof(V4) / 16;
      for (int e = threadIdx.x; e < ncopy * QV; e += blockDim.x)
        cp_async16(reinterpret_cast<unsigned char*>(TQ_b + b * kChunk) + 16 * e,
                   reinterpret_cast<const unsigned char*>(slot_tq + s0) + 16 * e);
      for (int e = threadIdx.x; e < ncopy / 4; e += blockDim.x)
        cp_async16(LB_b + b * kChunk + 4 * e, bins.lb + s0 + 4 * e);
      if (threadIdx.x == 0) cp_async_small<4>(CNT_b + b, bins.count + t);
      if (kFixed && threadIdx.x < kHQ / 4)
        cp_async16(HQ_b + b * kHQ + 4 * threadIdx.x, bins.hq + (int64_t)t * kHQ + 4 * threadIdx.x);
    }
    cp_async_commit();
  };

  auto take = [&](int* st, int3* so) {
    const int t = atomicAdd(&bins.ctrl[1], 1);
    *st = t;
    if (t < ntiles) {
      const int t2 = t % g.nt[2];
      const int t1 = (t / g.nt[2]) % g.nt[1];
      const int t0 = t / (g.nt[2] * g.nt[1]);
      *so = make_int3(t0 * g.T[0], t1 * g.T[1], t2 * g.T[2]);
    }
  };
  if (threadIdx.x == 0) {
    take(&s_first[0], &s_ofirst[0]);
    take(&s_first[1], &s_ofirst[1]);
  }
  {
    // clear the block once; every flush clears what it reads
    using Z = typename std::conditional<kFixed, int4, double2>::type;
    constexpr int nz = vol * (int)sizeof(A) / 16;
    Z* az = reinterpret_cast<Z*>(acc);
    const Z zero{};
    for (int e = threadIdx.x; e < nz; e += blockDim.x) az[e] = zero;
  }
  __syncthreads();
  int tile = s_first[0], nxt = s_first[1];
  int3 org = s_ofirst[0], nxt_o = s_ofirst[1];
  issue(tile, 0);
  issue(nxt, 1);

  for (int kt = 0; tile < ntiles; ++kt) {
    const int bf = kt & 1;
    if (threadIdx.x == 0) take(&s_ahead[bf], &s_oahead[bf]);
    cp_async_wait<1>();
    __syncthreads();  // tile's count and first atoms are in buffer bf
    V4* TQ = TQ_b + bf * kChunk;
    int* LB = LB_b + bf * kChunk;
    const int cnt_all = min(CNT_b[bf], bins.cap);
    if (threadIdx.x == 0) {
      // the gather reads the tile's atom count from tcount; the counter is zero again
      bins.tcount[tile] = cnt_all;
      bins.count[tile] = 0;
    }
    if (kFixed && threadIdx.x < kHQ) bins.hq[(int64_t)tile * kHQ + threadIdx.x] = 0.f;
    const int64_t s0 = (int64_t)tile * bins.cap;
    if (cnt_all > 0) {
      // fixed-point scale of this tile (FP32): a power of two, so scaling back is exact
      R scale = R(1), inv_scale = R(1);
      if constexpr (kFixed) {
        // A point (x0, x1, x2) of the block receives only from the atoms whose stencil base
        // b has x_2 - P < b_2 <= x_2, so the largest sum of |q| over such windows along axis
        // 2 (any b0, b1), times max |w|^3, bounds every partial sum.  HQ holds the tile's
        // sum |q| per base b2 (from the binning); lane x2 of warp 0 sums window x2.
        if (warp == 0) {
          const float* HQ = HQ_b + bf * kHQ;
          const int T2 = g.T[2];
          float mx = 0.f;
          for (int x2 = lane; x2 < E2; x2 += 32) {
            float sw = 0.f;
#pragma unroll
            for (int d2 = 0; d2 < P; ++d2) {
              const int b2 = x2 - d2;
              if (b2 >= 0 && b2 < T2) sw += HQ[b2];
            }
            mx = fmaxf(mx, sw);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          if (lane == 0) s_bound = mx;
        }
        __syncthreads();
        const float tot = s_bound;
        // with margin for the float sums
        const float bound = tot * g.wmax3 * 1.0001f + 1e-30f;
        int ex;
        frexpf(bound, &ex);  // bound < 2^ex
        ex = max(ex, -90);   // all-zero charges: any finite scale will do
        scale = ldexpf(1.f, 30 - ex);
        inv_scale = ldexpf(1.f, ex - 30);
      }
      for (int c0 = 0; c0 < cnt_all; c0 += kChunk) {
        const int cnt = min(kChunk, cnt_all - c0);
        if (c0 > 0) {
          // a tile with more atoms than a chunk: the later chunks are loaded here
          for (int a = threadIdx.x; a < cnt; a += blockDim.x) {
            TQ[a] = slot_tq[s0 + c0 + a];
            LB[a] = bins.lb[s0 + c0 + a];
          }
          __syncthreads();
        }
        if (a_t < NPA) {
          // coefficients of stencil point p_t (a small table, L1-resident): loaded here so
          // the registers are free in the other phases
          R cw[D + 1];
#pragma unroll
          for (int k = 0; k <= D; ++k) cw[k] = __ldg(wtab + k * P + p_t);
          for (int a = a_t; a < cnt; a += NPA) {
            const V4 v = TQ[a];
            const R w0 = horner_reg<R, D>(cw, v.x);
            const R w1 = horner_reg<R, D>(cw, v.y);
            const R w2 = horner_reg<R, D>(cw, v.z);
            R* Wa = W + a * RS + p_t;
            Wa[0] = w0;
            Wa[P] = w1 * (v.w * scale);
            Wa[2 * P] = w2;
          }
        }
        __syncthreads();
        // warp w takes a contiguous block of the chunk's atoms: the atoms the eight warps
        // add at the same time lie about cnt / 8 slots apart, not next to each other (the
        // binning fills slots molecule by molecule, whose stencils overlap)
        const int per = (cnt + kThreads / 32 - 1) / (kThreads / 32);
        const int aend = min(cnt, (warp + 1) * per);
        for (int a = warp * per; a < aend; ++a) {
          const R* Wa = W + a * RS;
          const unsigned base = acc_s + (unsigned)(local_base<S1, E3p>(LB[a]) * (int)sizeof(A));
          if constexpr (kFixed) {
            // the record's w0 as packed pairs straight from the 16-byte aligned record
            unsigned long long w0p[(P + 1) / 2];
            const unsigned long long* Wp = reinterpret_cast<const unsigned long long*>(Wa);
#pragma unroll
            for (int m = 0; m < (P + 1) / 2; ++m) w0p[m] = Wp[m];
#pragma unroll
            for (int m = 0; m < CM::MP; ++m) {
              const float pw = Wa[P + lc.j[m]] * Wa[2 * P + lc.k[m]];
              spread_column2<S1, P>(base + (unsigned)(lc.off[m] * (int)sizeof(A)), w0p,
                                    pack2(pw, pw),
                                    std::make_integer_sequence<int, (P + 1) / 2>{});
            }
          } else {
            R w0[P];
            load_record<R, P>(Wa, w0);
#pragma unroll
            for (int m = 0; m < CM::MP; ++m) {
              const R pw = Wa[P + lc.j[m]] * Wa[2 * P + lc.k[m]];
              spread_column<R, S1>(base + (unsigned)(lc.off[m] * (int)sizeof(A)), w0, pw,
                                   std::make_integer_sequence<int, P>{});
            }
          }
#pragma unroll
          for (int t = 0; t < CM::NG; ++t) {
            if (lc.tail_ok[t])
              red_fixed<0>(base + (unsigned)lc.tail_off[t],
                           Wa[lc.tail_i[t]] * (Wa[lc.tail_j[t]] * Wa[lc.tail_k[t]]));
          }
        }
        __syncthreads();
      }

      // add the padded block into the periodic global grid, clearing it
      const int o0 = org.x, o1 = org.y, o2 = org.z;
      bool flushed = false;
      if constexpr (kFixed) {
        if (g.vec4) {
          const int E2v = (E2 + 3) >> 2;
          const int nflush = E0 * E1 * E2v;
          for (int e = threadIdx.x; e < nflush; e += blockDim.x) {
            const int ab = fast_div(e, g.div_E2v);
            const int c4 = e - ab * E2v;
            const int a = ab / E1;
            const int b = ab - a * E1;
            if (b >= g.E[1]) continue;
            int* src = acc + a * S1 + b * E3p + 4 * c4;
            const int4 iv = make_int4(src[0], src[1], src[2], src[3]);
            if (iv.x | iv.y | iv.z | iv.w) {
              src[0] = 0;
              src[1] = 0;
              src[2] = 0;
              src[3] = 0;
              const int gi = wrap3(o0 + a, g.M[0]);
              const int gj = wrap3(o1 + b, g.M[1]);
              const int gk = wrap3(o2 + 4 * c4, g.M[2]);
              red_add4(grid + ((int64_t)gi * g.M[1] + gj) * g.M[2] + gk, (float)iv.x * inv_scale,
                       (float)iv.y * inv_scale, (float)iv.z * inv_scale, (float)iv.w * inv_scale);
            }
          }
          flushed = true;
        }
      }
      if (!flushed) {
        const int E1r = g.E[1];
        const int nflush = E0 * E1r * E2;
        for (int e = threadIdx.x; e < nflush; e += blockDim.x) {
          const int c = e % E2;
          const int ab = e / E2;
          const int b = ab % E1r;
          const int a = ab / E1r;
          A* src = acc + a * S1 + b * E3p + c;
          const A av = *src;
          if (av != A(0)) {
            *src = A(0);
            const R val = kFixed ? R((float)av * (float)inv_scale) : R(av);
            const int gi = wrap_index(o0 + a, g.M[0]);
            const int gj = wrap_index(o1 + b, g.M[1]);
            const int gk = wrap_index(o2 + c, g.M[2]);
            atomicAdd(&grid[((int64_t)gi * g.M[1] + gj) * g.M[2] + gk], val);
          }
        }
      }
    }
    __syncthreads();  // the block is read out and cleared; buffer bf is free
    const int nn = s_ahead[bf];
    const int3 nn_o = s_oahead[bf];
    issue(nn, bf);
    tile = nxt;
    org = nxt_o;
    nxt = nn;
    nxt_o = nn_o;
  }
  cp_async_wait<0>();
  __syncthreads();

  // atoms past their tile's capacity: one warp per atom, window values in the warp's part
  // of the record area, global atomics with periodic wrap
  {
    const int novf = bins.ctrl[0];
    R* Ww = W + warp * (3 * kMaxP);
    const V4* otq = static_cast<const V4*>(bins.otq);
    for (;;) {
      int o = 0;
      if (lane == 0) o = atomicAdd(&bins.ctrl[2], 1);
      o = __shfl_sync(0xffffffffu, o, 0);
      if (o >= novf) break;
      const V4 v = otq[o];
      const int b0 = bins.ob[3 * o], b1 = bins.ob[3 * o + 1], b2 = bins.ob[3 * o + 2];
      for (int e = lane; e < 3 * P; e += 32) {
        const int d = e / P, pp = e - d * P;
        const R tau = tq_comp<R>(v, d) - R(0.5);
        R w = wtab[D * P + pp];
        for (int k = D - 1; k >= 0; --k) w = fma(w, tau, wtab[k * P + pp]);
        Ww[e] = w;
      }
      __syncwarp();
      for (int l = lane; l < P * P * P; l += 32) {
        const int i = l / (P * P), r = l - i * (P * P), j = r / P, k = r - j * P;
        const R val = v.w * Ww[i] * Ww[P + j] * Ww[2 * P + k];
        const int gi = wrap_index(b0 + i, g.M[0]);
        const int gj = wrap_index(b1 + j, g.M[1]);
        const int gk = wrap_index(b2 + k, g.M[2]);
        atomicAdd(&grid[((int64_t)gi * g.M[1] + gj) * g.M[2] + gk], val);
      }
      __syncwarp();
    }
  }
  // the overflow count passes to the gather; the spread's counters are zero again
  last_cta_resets(bins.ctrl, 3, 1, 3, 0, 4);
}

// ---------------------------------------------------------------------------------------
// Radial psi_0 / psi_0' on x in [0, 1] by kRadialPieces Horner pieces in (x - centre).
template <typename R>
__device__ __forceinline__ void radial_eval(const R* __restrict__ rt, int rdeg, R x, R* psi,
                                            R* dpsi) {
  int piece = (int)(x * R(kRadialPieces));
  piece = piece < 0 ? 0 : (piece >= kRadialPieces ? kRadialPieces - 1 : piece);
  const R tau = x - (R(piece) + R(0.5)) / R(kRadialPieces);
  const R* a = rt + piece * (rdeg + 1);
  const R* b = rt + (kRadialPieces + piece) * (rdeg + 1);
  R u = a[rdeg], w = b[rdeg];
  for (int k = rdeg - 1; k >= 0; --k) {
    u = fma(u, tau, a[k]);
    w = fma(w, tau, b[k]);
  }
  *psi = u;
  *dpsi = w;
}

template <typename R>
__device__ __forceinline__ R bvec(const ScaleGeom& s, int i);
template <>
__device__ __forceinline__ float bvec<float>(const ScaleGeom& s, int i) {
  return s.bf[i];
}
template <>
__device__ __forceinline__ double bvec<double>(const ScaleGeom& s, int i) {
  return s.b[i];
}

template <typename R>
struct ScaleConst {
  R K2, x_per_k, A, scale;
  __device__ __forceinline__ explicit ScaleConst(const ScaleGeom& s) {
    if constexpr (std::is_same<R, float>::value) {
      K2 = s.K2f;
      x_per_k = s.x_per_kf;
      A = s.Af;
      scale = s.scalef;
    } else {
      K2 = s.K2;
      x_per_k = s.x_per_k;
      A = s.A;
      scale = s.scale;
    }
  }
};

// ---------------------------------------------------------------------------------------
// The transform along the first grid axis, fused with the scaling and the reduction
// (eqs. (UF) and (WF)).  cuFFT transforms the planes i0 = const over (i1, i2) (R2C along
// i2, then along i1); what is left of the 3D transform is an FFT of length M0 along every
// column (i1, i2) of the [M0][M1][H2] half spectrum.  A CTA takes NC consecutive columns
// (consecutive in memory, so each row i0 is one contiguous segment), keeps them in shared
// memory as buf[i0][c] and runs
//   FWD: the forward transform along i0 (mixed-radix Stockham passes);
//   the sums of eqs. (UF) / (WF) over the sphere |k| <= K, and with INV the scaling of
//        every mode by G(k) = F^(k) / w^(k)^2;
//   INV: the inverse transform along i0 of the scaled modes.
// Without FWD the columns hold the full 3D spectrum X already (the energy and pressure
// path and the kept spectrum); without INV nothing is written.  Column groups come in the
// order order[blockIdx]: the first nactive hold every column whose line through k may
// enter the sphere (colact = 1, decided on the host from the cell).  The grid is those
// nactive CTAs; with INV they write their columns to out, whose other columns (all of
// whose modes scale to zero) the caller has cleared.  FP32: compensated FP32 sums (about 48 significant bits);
// FP64: plain FP64.  Per-CTA sums go to partials; k_xsum adds them up.

// DIT Stockham pass over buf[i0][c] (Govindaraju et al., SC'08, restated for mixed radix):
// butterfly j < M0 / RAD, k = j mod Ns, reads in[j + t M0 / RAD], multiplies by
// w^(t k M0 / (Ns RAD)) (w = e^{-2 pi i / M0}; conjugate for the inverse), takes the
// RAD-point DFT and writes out[(j - k) RAD + k + t Ns]; Ns is the product of the radices
// of the passes before.
template <typename R>
__device__ __forceinline__ typename Cplx<R>::T cmk(R x, R y) {
  typename Cplx<R>::T z;
  z.x = x;
  z.y = y;
  return z;
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) {
  a.x += b.x;
  a.y += b.y;
  return a;
}
template <typename C>
__device__ __forceinline__ C csub(C a, C b) {
  a.x -= b.x;
  a.y -= b.y;
  return a;
}
// a * w (SIGN < 0) or a * conj(w) (SIGN > 0)
template <int SIGN, typename C>
__device__ __forceinline__ C ctw(C a, C w) {
  C z;
  if constexpr (SIGN < 0) {
    z.x = a.x * w.x - a.y * w.y;
    z.y = a.x * w.y + a.y * w.x;
  } else {
    z.x = a.x * w.x + a.y * w.y;
    z.y = a.y * w.x - a.x * w.y;
  }
  return z;
}
// a * (SIGN i)
template <int SIGN, typename C>
__device__ __forceinline__ C crot(C a) {
  C z;
  if constexpr (SIGN < 0) {
    z.x = a.y;
    z.y = -a.x;
  } else {
    z.x = -a.y;
    z.y = a.x;
  }
  return z;
}

template <int SIGN, typename C>
__device__ __forceinline__ void dft4(C& a, C& b, C& c, C& d) {
  const C s0 = cadd(a, c), d0 = csub(a, c), s1 = cadd(b, d), d1 = crot<SIGN>(csub(b, d));
  a = cadd(s0, s1);
  c = csub(s0, s1);
  b = cadd(d0, d1);
  d = csub(d0, d1);
}

// RAD-point DFT in registers, y_u = sum_t v_t e^{SIGN 2 pi i u t / RAD}.  RAD = 3, 5, 7 take
// their roots from the table (root m at index m M0 / RAD).
template <typename R, int RAD, int SIGN>
__device__ __forceinline__ void dft_reg(typename Cplx<R>::T (&v)[RAD],
                                        const typename Cplx<R>::T* tw, int M0) {
  using C = typename Cplx<R>::T;
  if constexpr (RAD == 2) {
    const C a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  } else if constexpr (RAD == 4) {
    dft4<SIGN>(v[0], v[1], v[2], v[3]);
  } else if constexpr (RAD == 8) {
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<SIGN>(e0, e1, e2, e3);
    dft4<SIGN>(o0, o1, o2, o3);
    const R h = R(0.70710678118654752440);  // 1 / sqrt(2)
    // o_u *= e^{SIGN 2 pi i u / 8}
    o1 = cmk<R>(h * (o1.x - SIGN * o1.y), h * (o1.y + SIGN * o1.x));
    o2 = crot<SIGN>(o2);
    o3 = cmk<R>(h * (-o3.x - SIGN * o3.y), h * (-o3.y + SIGN * o3.x));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
  } else {
    C w[RAD];
    const int step = M0 / RAD;
#pragma unroll
    for (int m = 0; m < RAD; ++m) w[m] = tw[m * step];
    C y[RAD];
#pragma unroll
    for (int u = 0; u < RAD; ++u) {
      C a = v[0];
#pragma unroll
      for (int t = 1; t < RAD; ++t) {
        const C z = ctw<SIGN>(v[t], w[(u * t) % RAD]);
        a.x += z.x;
        a.y += z.y;
      }
      y[u] = a;
    }
#pragma unroll
    for (int u = 0; u < RAD; ++u) v[u] = y[u];
  }
}

template <typename R, int RAD, int SIGN>
__device__ __forceinline__ void xpass(const typename Cplx<R>::T* in, typename Cplx<R>::T* out,
                                      const typename Cplx<R>::T* tw, int M0, int lognc,
                                      int Ns, unsigned int ns_magic) {
  using C = typename Cplx<R>::T;
  const int L = M0 / RAD;
  const int stride = L / Ns;  // M0 / (Ns RAD)
  const int ncm = (1 << lognc) - 1;
  const int nb = L << lognc;
  const int Lnc = L << lognc, Nsnc = Ns << lognc;  // element strides of inputs and outputs
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int c = b & ncm, j = b >> lognc;
    const int k = Ns == 1 ? 0 : j - fast_div(j, ns_magic) * Ns;
    C v[RAD];
    const C* src = in + b;  // b = (j << lognc) + c
#pragma unroll
    for (int t = 0; t < RAD; ++t) v[t] = src[t * Lnc];
    if (k > 0) {
      const int ks = k * stride;
      const C* w = tw + ks;
#pragma unroll
      for (int t = 1; t < RAD; ++t) v[t] = ctw<SIGN>(v[t], w[(t - 1) * ks]);
    }
    dft_reg<R, RAD, SIGN>(v, tw, M0);
    C* dst = out + (((j - k) * RAD + k) << lognc) + c;
#pragma unroll
    for (int t = 0; t < RAD; ++t) dst[t * Nsnc] = v[t];
  }
}

// A pass of a prime radix p > 7: one output per thread, p products each.
template <typename R, int SIGN>
__device__ __forceinline__ void xpass_any(const typename Cplx<R>::T* in,
                                          typename Cplx<R>::T* out,
                                          const typename Cplx<R>::T* tw, int M0, int lognc,
                                          int Ns, unsigned int ns_magic, int p) {
  using C = typename Cplx<R>::T;
  const int L = M0 / p;
  const int stride = L / Ns;
  const int ncm = (1 << lognc) - 1;
  const int n = M0 << lognc;
  for (int o = threadIdx.x; o < n; o += blockDim.x) {
    const int c = o & ncm, r = o >> lognc;
    const int u = r / L, j = r - u * L;
    const int k = Ns == 1 ? 0 : j - fast_div(j, ns_magic) * Ns;
    C a = cmk<R>(R(0), R(0));
    for (int t = 0; t < p; ++t) {
      int idx = t * k * stride + ((u * t) % p) * L;
      if (idx >= M0) idx -= M0;
      const C z = ctw<SIGN>(in[((j + t * L) << lognc) + c], tw[idx]);
      a.x += z.x;
      a.y += z.y;
    }
    out[(((j - k) * p + k + u * Ns) << lognc) + c] = a;
  }
}

// All passes of one direction; returns the buffer that holds the result.
template <typename R, int SIGN>
__device__ __forceinline__ typename Cplx<R>::T* xfft_lines(typename Cplx<R>::T* a,
                                                           typename Cplx<R>::T* b,
                                                           const typename Cplx<R>::T* tw,
                                                           const XGeom& x) {
  int Ns = 1;
  for (int s = 0; s < x.npass; ++s) {
    const int rad = x.radix[s];
    const unsigned int mg = x.ns_magic[s];
    switch (rad) {
      case 8: xpass<R, 8, SIGN>(a, b, tw, x.M0, x.lognc, Ns, mg); break;
      case 4: xpass<R, 4, SIGN>(a, b, tw, x.M0, x.lognc, Ns, mg); break;
      case 2: xpass<R, 2, SIGN>(a, b, tw, x.M0, x.lognc, Ns, mg); break;
      case 3: xpass<R, 3, SIGN>(a, b, tw, x.M0, x.lognc, Ns, mg); break;
      case 5: xpass<R, 5, SIGN>(a, b, tw, x.M0, x.lognc, Ns, mg); break;
      case 7: xpass<R, 7, SIGN>(a, b, tw, x.M0, x.lognc, Ns, mg); break;
      default: xpass_any<R, SIGN>(a, b, tw, x.M0, x.lognc, Ns, mg, rad); break;
    }
    Ns *= rad;
    __syncthreads();
    typename Cplx<R>::T* t = a;
    a = b;
    b = t;
  }
  return a;
}

// ---------------------------------------------------------------------------------------
// Line transforms of the plane kernels: the same Stockham passes as xpass, over nc (odd)
// columns with element (j, c) at j * nc + c; c = b mod nc by magic division.
template <typename R, int RAD, int SIGN>
__device__ __forceinline__ void lpass(const typename Cplx<R>::T* in, typename Cplx<R>::T* out,
                                      const typename Cplx<R>::T* tw, const LineFFT& f, int Ns,
                                      unsigned int ns_magic) {
  using C = typename Cplx<R>::T;
  const int N = f.n, nc = f.nc;
  const int L = N / RAD;
  const int stride = L / Ns;
  const int nb = L * nc;
  const int Lnc = L * nc, Nsnc = Ns * nc;  // element strides of the RAD inputs and outputs
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    // b = j nc + c: input t of butterfly j in column c is in[b + t L nc]
    const int j = fast_div(b, f.nc_magic);
    const int c = b - j * nc;
    const int k = Ns == 1 ? 0 : j - fast_div(j, ns_magic) * Ns;
    C v[RAD];
    const C* src = in + b;
#pragma unroll
    for (int t = 0; t < RAD; ++t) v[t] = src[t * Lnc];
    if (k > 0) {
      const int ks = k * stride;
      const C* w = tw + ks;
#pragma unroll
      for (int t = 1; t < RAD; ++t) v[t] = ctw<SIGN>(v[t], w[(t - 1) * ks]);
    }
    dft_reg<R, RAD, SIGN>(v, tw, N);
    C* dst = out + ((j - k) * RAD + k) * nc + c;
#pragma unroll
    for (int t = 0; t < RAD; ++t) dst[t * Nsnc] = v[t];
  }
}

template <typename R, int SIGN>
__device__ __forceinline__ void lpass_any(const typename Cplx<R>::T* in,
                                          typename Cplx<R>::T* out,
                                          const typename Cplx<R>::T* tw, const LineFFT& f,
                                          int Ns, unsigned int ns_magic, int p) {
  using C = typename Cplx<R>::T;
  const int N = f.n, nc = f.nc;
  const int L = N / p;
  const int stride = L / Ns;
  const int n = N * nc;
  for (int o = threadIdx.x; o < n; o += blockDim.x) {
    const int r = fast_div(o, f.nc_magic);
    const int c = o - r * nc;
    const int u = r / L, j = r - u * L;
    const int k = Ns == 1 ? 0 : j - fast_div(j, ns_magic) * Ns;
    C a = cmk<R>(R(0), R(0));
    for (int t = 0; t < p; ++t) {
      int idx = t * k * stride + ((u * t) % p) * L;
      if (idx >= N) idx -= N;
      const C z = ctw<SIGN>(in[(j + t * L) * nc + c], tw[idx]);
      a.x += z.x;
      a.y += z.y;
    }
    out[((j - k) * p + k + u * Ns) * nc + c] = a;
  }
}

// All passes of one line transform; returns the buffer that holds the result.
template <typename R, int SIGN>
__device__ __forceinline__ typename Cplx<R>::T* lfft_lines(typename Cplx<R>::T* a,
                                                           typename Cplx<R>::T* b,
                                                           const typename Cplx<R>::T* tw,
                                                           const LineFFT& f) {
  int Ns = 1;
  for (int s = 0; s < f.npass; ++s) {
    const int rad = f.radix[s];
    const unsigned int mg = f.ns_magic[s];
    switch (rad) {
      case 8: lpass<R, 8, SIGN>(a, b, tw, f, Ns, mg); break;
      case 4: lpass<R, 4, SIGN>(a, b, tw, f, Ns, mg); break;
      case 2: lpass<R, 2, SIGN>(a, b, tw, f, Ns, mg); break;
      case 3: lpass<R, 3, SIGN>(a, b, tw, f, Ns, mg); break;
      case 5: lpass<R, 5, SIGN>(a, b, tw, f, Ns, mg); break;
      case 7: lpass<R, 7, SIGN>(a, b, tw, f, Ns, mg); break;
      default: lpass_any<R, SIGN>(a, b, tw, f, Ns, mg, rad); break;
    }
    Ns *= rad;
    __syncthreads();
    typename Cplx<R>::T* t = a;
    a = b;
    b = t;
  }
  return a;
}

// ---------------------------------------------------------------------------------------
// Line transforms of lengths known at compile time (the common grid sizes): the same
// Stockham passes with the pass lengths, strides and twiddle steps as constants, and the
// radix-3 and radix-5 butterflies from their closed forms.
struct CPlan {
  int npass;
  int radix[kMaxPass];
};
__host__ __device__ constexpr CPlan cplan(int n) {
  CPlan p{0, {}};
  while (n % 8 == 0) {
    p.radix[p.npass++] = 8;
    n /= 8;
  }
  if (n % 4 == 0) {
    p.radix[p.npass++] = 4;
    n /= 4;
  }
  if (n % 2 == 0) {
    p.radix[p.npass++] = 2;
    n /= 2;
  }
  while (n % 3 == 0) {
    p.radix[p.npass++] = 3;
    n /= 3;
  }
  while (n % 5 == 0) {
    p.radix[p.npass++] = 5;
    n /= 5;
  }
  if (n > 1) p.npass = -1;  // other factors: no compile-time plan
  return p;
}

// RAD-point DFT y_u = sum_t v_t e^{SIGN 2 pi i u t / RAD} for RAD = 2, 4, 8, 3, 5.
// Radix 3: with w = -1/2 + i SIGN sqrt(3)/2, y_1,2 = a - (b + c)/2 +- i SIGN sqrt(3)/2 (b - c).
// Radix 5: with s1 = v1 + v4, d1 = v1 - v4, s2 = v2 + v3, d2 = v2 - v3 and th = 2 pi / 5,
//   y_1,4 = v0 + cos(th) s1 + cos(2 th) s2 +- i SIGN (sin(th) d1 + sin(2 th) d2),
//   y_2,3 = v0 + cos(2 th) s1 + cos(th) s2 +- i SIGN (sin(2 th) d1 - sin(th) d2).
template <typename R, int RAD, int SIGN>
__device__ __forceinline__ void dft_fixed(typename Cplx<R>::T (&v)[RAD]) {
  using C = typename Cplx<R>::T;
  if constexpr (RAD == 2 || RAD == 4 || RAD == 8) {
    dft_reg<R, RAD, SIGN>(v, nullptr, 0);
  } else if constexpr (RAD == 3) {
    const R h = R(0.866025403784438646763723170753);  // sqrt(3) / 2
    const C t1 = cadd(v[1], v[2]);
    const C t2 = cmk<R>(v[0].x - R(0.5) * t1.x, v[0].y - R(0.5) * t1.y);
    const C d = cmk<R>(R(SIGN) * h * (v[1].x - v[2].x), R(SIGN) * h * (v[1].y - v[2].y));
    v[0] = cadd(v[0], t1);
    v[1] = cmk<R>(t2.x - d.y, t2.y + d.x);
    v[2] = cmk<R>(t2.x + d.y, t2.y - d.x);
  } else if constexpr (RAD == 5) {
    const R c1 = R(0.309016994374947424102293417183), c2 = R(-0.809016994374947424102293417183);
    const R s1 = R(0.951056516295153572116439333379), s2 = R(0.587785252292473129168705954639);
    const C p1 = cadd(v[1], v[4]), m1 = csub(v[1], v[4]);
    const C p2 = cadd(v[2], v[3]), m2 = csub(v[2], v[3]);
    const C a1 = cmk<R>(v[0].x + c1 * p1.x + c2 * p2.x, v[0].y + c1 * p1.y + c2 * p2.y);
    const C a2 = cmk<R>(v[0].x + c2 * p1.x + c1 * p2.x, v[0].y + c2 * p1.y + c1 * p2.y);
    const C b1 = cmk<R>(R(SIGN) * (s1 * m1.x + s2 * m2.x), R(SIGN) * (s1 * m1.y + s2 * m2.y));
    const C b2 = cmk<R>(R(SIGN) * (s2 * m1.x - s1 * m2.x), R(SIGN) * (s2 * m1.y - s1 * m2.y));
    v[0] = cadd(v[0], cadd(p1, p2));
    v[1] = cmk<R>(a1.x - b1.y, a1.y + b1.x);  // a1 + i b1
    v[4] = cmk<R>(a1.x + b1.y, a1.y - b1.x);  // a1 - i b1
    v[2] = cmk<R>(a2.x - b2.y, a2.y + b2.x);
    v[3] = cmk<R>(a2.x + b2.y, a2.y - b2.x);
  }
}

template <typename R, int RAD, int SIGN, int N, int NS>
__device__ __forceinline__ void lpass_fixed(const typename Cplx<R>::T* in, typename Cplx<R>::T* out,
                                            const typename Cplx<R>::T* tw, int nc,
                                            unsigned int nc_magic) {
  using C = typename Cplx<R>::T;
  constexpr int L = N / RAD;
  constexpr int stride = L / NS;
  const int nb = L * nc;
  const int Lnc = L * nc, Nsnc = NS * nc;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int j = fast_div(b, nc_magic);
    const int c = b - j * nc;
    const int k = NS == 1 ? 0 : j % NS;
    C v[RAD];
    const C* src = in + b;
#pragma unroll
    for (int t = 0; t < RAD; ++t) v[t] = src[t * Lnc];
    if (k > 0) {
      const C* w = tw + k * stride;
#pragma unroll
      for (int t = 1; t < RAD; ++t) v[t] = ctw<SIGN>(v[t], w[(t - 1) * k * stride]);
    }
    dft_fixed<R, RAD, SIGN>(v);
    C* dst = out + ((j - k) * RAD + k) * nc + c;
#pragma unroll
    for (int t = 0; t < RAD; ++t) dst[t * Nsnc] = v[t];
  }
}

template <typename R, int SIGN, int N, int S, int NS>
__device__ __forceinline__ typename Cplx<R>::T* lfft_fixed(typename Cplx<R>::T* a,
                                                           typename Cplx<R>::T* b,
                                                           const typename Cplx<R>::T* tw, int nc,
                                                           unsigned int nc_magic) {
  constexpr CPlan pl = cplan(N);
  if constexpr (S >= pl.npass) {
    return a;
  } else {
    constexpr int RAD = pl.radix[S];
    lpass_fixed<R, RAD, SIGN, N, NS>(a, b, tw, nc, nc_magic);
    __syncthreads();
    return lfft_fixed<R, SIGN, N, S + 1, NS * RAD>(b, a, tw, nc, nc_magic);
  }
}

// The line transform of f: a compile-time version for the common lengths, else the
// generic passes.
template <typename R, int SIGN>
__device__ __forceinline__ typename Cplx<R>::T* lfft_any(typename Cplx<R>::T* a,
                                                         typename Cplx<R>::T* b,
                                                         const typename Cplx<R>::T* tw,
                                                         const LineFFT& f) {
  switch (f.n) {
    case 24: return lfft_fixed<R, SIGN, 24, 0, 1>(a, b, tw, f.nc, f.nc_magic);
    case 32: return lfft_fixed<R, SIGN, 32, 0, 1>(a, b, tw, f.nc, f.nc_magic);
    case 64: return lfft_fixed<R, SIGN, 64, 0, 1>(a, b, tw, f.nc, f.nc_magic);
    case 72: return lfft_fixed<R, SIGN, 72, 0, 1>(a, b, tw, f.nc, f.nc_magic);
    case 96: return lfft_fixed<R, SIGN, 96, 0, 1>(a, b, tw, f.nc, f.nc_magic);
    case 128: return lfft_fixed<R, SIGN, 128, 0, 1>(a, b, tw, f.nc, f.nc_magic);
    case 160: return lfft_fixed<R, SIGN, 160, 0, 1>(a, b, tw, f.nc, f.nc_magic);
    case 256: return lfft_fixed<R, SIGN, 256, 0, 1>(a, b, tw, f.nc, f.nc_magic);
    default: return lfft_lines<R, SIGN>(a, b, tw, f);
  }
}

// Sums of 8 values over the 32 lanes of a warp in a fixed order.  Each of the first three
// levels halves the values a lane keeps and sends the other half to its partner, so lane l
// ends with the warp total of value c(l) = 4 ((l >> 4) & 1) + 2 ((l >> 3) & 1) + ((l >> 2)
// & 1): 9 shuffle-and-add steps instead of 8 x 5.
__device__ __forceinline__ DF shfl_xor(const DF& a, int o) {
  DF r;
  r.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
  r.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
  return r;
}
__device__ __forceinline__ double shfl_xor(double a, int o) {
  return __shfl_xor_sync(0xffffffffu, a, o);
}
__device__ __forceinline__ void acc_add(DF& a, const DF& b) { a.add(b); }
__device__ __forceinline__ void acc_add(double& a, double b) { a += b; }
__device__ __forceinline__ int sum8_slot(int lane) {
  return 4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1);
}
template <typename A>
__device__ __forceinline__ A warp_sum8(const A (&v)[8]) {
  const int lane = threadIdx.x & 31;
  A w4[4], w2[2], w1;
  {
    const bool up = (lane & 16) != 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      w4[i] = up ? v[4 + i] : v[i];
      acc_add(w4[i], shfl_xor(up ? v[i] : v[4 + i], 16));
    }
  }
  {
    const bool up = (lane & 8) != 0;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      w2[i] = up ? w4[2 + i] : w4[i];
      acc_add(w2[i], shfl_xor(up ? w4[i] : w4[2 + i], 8));
    }
  }
  {
    const bool up = (lane & 4) != 0;
    w1 = up ? w2[1] : w2[0];
    acc_add(w1, shfl_xor(up ? w2[0] : w2[1], 4));
  }
  acc_add(w1, shfl_xor(w1, 2));
  acc_add(w1, shfl_xor(w1, 1));
  return w1;
}

// The 7 reduction components (U_F and W_F xx yy zz xy xz yz) of a CTA in a fixed order:
// warp_sum8, then threads j < 7 add the NW warp totals of component j in warp order.
template <typename A, int NW>
__device__ __forceinline__ A cta_sum7(const A (&acc)[7], A (*red)[NW]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  A v[8];
#pragma unroll
  for (int j = 0; j < 7; ++j) v[j] = acc[j];
  v[7] = A{};
  const A t = warp_sum8(v);
  const int c = sum8_slot(lane);
  if ((lane & 3) == 0 && c < 7) red[c][wid] = t;
  __syncthreads();
  A r{};
  if (threadIdx.x < 7)
    for (int w = 0; w < NW; ++w) acc_add(r, red[threadIdx.x][w]);
  return r;
}

// Final sums in a fixed order, one CTA launched after k_xfft (on a branch of its own in the
// step graph): accum[0..6] from the per-CTA partials of k_xfft (component j at
// partials[j * nblk + b]); accum[7..9] (sum q, sum q^2, skipped atoms) from the binning
// partials (3 compensated pairs per k_bin block).
template <typename R>
__global__ void __launch_bounds__(kThreads) k_xsum(const double* __restrict__ partials, int nblk,
                                                   const float2* __restrict__ bin_part, int nbin,
                                                   double* __restrict__ accum) {
  using A = typename std::conditional<std::is_same<R, double>::value, double, DF>::type;
  __shared__ A red[7][kThreads / 32];
  __shared__ DF redb[7][kThreads / 32];
  {
    DF sb[7];
#pragma unroll 4
    for (int b = threadIdx.x; b < nbin; b += blockDim.x) {
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float2 v = bin_part[3 * b + j];
        DF y;
        y.hi = v.x;
        y.lo = v.y;
        sb[j].add(y);
      }
    }
    const DF t = cta_sum7<DF, kThreads / 32>(sb, redb);
    if (threadIdx.x < 3) accum[7 + threadIdx.x] = (double)t.hi + (double)t.lo;
  }
  A s[7];
#pragma unroll
  for (int j = 0; j < 7; ++j) s[j] = A{};
#pragma unroll 4
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      if constexpr (std::is_same<R, double>::value) {
        s[j] += partials[(size_t)j * nblk + b];
      } else {
        const float2 v = reinterpret_cast<const float2*>(partials)[(size_t)j * nblk + b];
        DF y;
        y.hi = v.x;
        y.lo = v.y;
        s[j].add(y);
      }
    }
  }
  const A t = cta_sum7<A, kThreads / 32>(s, red);
  if (threadIdx.x < 7) {
    if constexpr (std::is_same<R, double>::value)
      accum[threadIdx.x] = t;
    else
      accum[threadIdx.x] = (double)t.hi + (double)t.lo;
  }
}

template <typename R, bool FWD, bool INV>
__global__ void __launch_bounds__(kXThreads, std::is_same<R, float>::value ? 2 : 1) k_xfft(const typename Cplx<R>::T* __restrict__ spec,
                                                   typename Cplx<R>::T* __restrict__ out,
                                                   XGeom x, ScaleGeom s,
                                                   const typename Cplx<R>::T* __restrict__ twg,
                                                   const R* __restrict__ invw2,
                                                   const R* __restrict__ radtab,
                                                   double* __restrict__ partials,
                                                   const int* __restrict__ order,
                                                   const unsigned char* __restrict__ colact,
                                                   int nactive) {
  using C = typename Cplx<R>::T;
  constexpr bool kD = std::is_same<R, double>::value;
  using Acc = typename std::conditional<kD, double, DF>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M0 = x.M0, lognc = x.lognc, NC = 1 << lognc;
  const int nrt = 2 * kRadialPieces * (s.rdeg + 1);
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf0 = tw + M0;
  C* buf1 = buf0 + (M0 << lognc);
  R* iw0 = reinterpret_cast<R*>(buf1 + (M0 << lognc));  // 1 / w0^2 along the column
  R* rt = iw0 + M0;                                    // radial polynomials
  // per column: k of (0, m1, m2), 1 / (w1^2 w2^2) times the Hermitian weight, m1, m2, flags
  __shared__ R ck[3][32], cw[32], cg[32];
  __shared__ int cm1[32], cm2[32], cflag[32];
  const int f0 = order[blockIdx.x] * NC;
  const int total = M0 << lognc;
  const int64_t rowst = x.ncol;  // elements between rows i0 and i0 + 1
  const ScaleConst<R> sc(s);

  if (threadIdx.x < NC) {
    const int c = threadIdx.x, f = f0 + c;
    int flag = 0;
    if (f < x.ncol) {
      const int b1 = f / x.nb2, i2 = f - b1 * x.nb2;
      const int m1 = (2 * b1 <= x.nb1) ? b1 : b1 - x.nb1;
      const int i1 = m1 < 0 ? m1 + s.M[1] : m1;
      const int m2 = i2;
      flag = colact[f] ? 3 : 1;  // a column of the spectrum; 3: its line may meet the sphere
      const R f1 = R(m1), f2 = R(m2);
      ck[0][c] = f1 * bvec<R>(s, 3) + f2 * bvec<R>(s, 6);
      ck[1][c] = f1 * bvec<R>(s, 4) + f2 * bvec<R>(s, 7);
      ck[2][c] = f1 * bvec<R>(s, 5) + f2 * bvec<R>(s, 8);
      const bool single = (i2 == 0) || ((s.M[2] & 1) == 0 && 2 * i2 == s.M[2]);
      cg[c] = invw2[s.M[0] + i1] * invw2[s.M[0] + s.M[1] + i2];
      cw[c] = (single ? R(1) : R(2)) * cg[c];
      cm1[c] = m1;
      cm2[c] = m2;
    }
    cflag[c] = flag;
  }
  for (int e = threadIdx.x; e < M0; e += blockDim.x) {
    tw[e] = twg[e];
    iw0[e] = invw2[e];
  }
  for (int e = threadIdx.x; e < nrt; e += blockDim.x) rt[e] = radtab[e];
  Acc acc[7];
  if constexpr (kD)
    for (int j = 0; j < 7; ++j) acc[j] = 0.0;
  {
    // the columns into shared memory, kU loads in flight per thread
    constexpr int kU = 4;
    for (int e0 = threadIdx.x; e0 < total; e0 += kU * blockDim.x) {
      C v[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = e0 + u * blockDim.x;
        const int f = f0 + (e & (NC - 1));
        v[u] = (e < total && f < x.ncol) ? spec[(int64_t)(e >> lognc) * rowst + f]
                                         : cmk<R>(R(0), R(0));
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < total) buf0[e] = v[u];
      }
    }
    __syncthreads();
    C* cur = buf0;
    C* oth = buf1;
    if (FWD) {
      cur = xfft_lines<R, -1>(buf0, buf1, tw, x);
      oth = cur == buf0 ? buf1 : buf0;
    }
    // scaling and sums; uniform trip count per warp (the FP64 boundary test is voted)
    for (int e0 = 0; e0 < total; e0 += blockDim.x) {
      const int e = e0 + threadIdx.x;
      const bool ok = e < total;
      const int c = e & (NC - 1), i0 = e >> lognc;
      const int m0 = (2 * i0 <= M0) ? i0 : i0 - M0;
      bool inside = ok && cflag[c] == 3 && abs(m0) <= s.mmax[0] && (m0 | cm1[c] | cm2[c]) != 0;
      R kx = R(0), ky = R(0), kz = R(0), k2 = R(0);
      if (inside) {
        const R f0r = R(m0);
        kx = f0r * bvec<R>(s, 0) + ck[0][c];
        ky = f0r * bvec<R>(s, 1) + ck[1][c];
        kz = f0r * bvec<R>(s, 2) + ck[2][c];
        k2 = kx * kx + ky * ky + kz * kz;
      }
      // the in-sphere decision is an FP64 one (as in the FP64 oracle); FP32 decides only
      // away from the boundary
      const bool near = inside && (kD || fabs(k2 - sc.K2) <= R(1e-5) * sc.K2);
      if (__any_sync(0xffffffffu, near)) {
        if (near) {
          const int m1 = cm1[c], m2 = cm2[c];
          const double dx = m0 * s.b[0] + m1 * s.b[3] + m2 * s.b[6];
          const double dy = m0 * s.b[1] + m1 * s.b[4] + m2 * s.b[7];
          const double dz = m0 * s.b[2] + m1 * s.b[5] + m2 * s.b[8];
          inside = dx * dx + dy * dy + dz * dz <= s.K2;
        }
      }
      if (!kD && !near && inside) inside = k2 <= sc.K2;
      if (!ok) continue;
      if (!inside) {
        if (INV) cur[e] = cmk<R>(R(0), R(0));
        continue;
      }
      const C X = cur[e];
      const R iw = iw0[i0] * cw[c];
      const R kmag = sqrt(k2);
      const R xa = kmag * sc.x_per_k;
      R psi, dpsi;
      radial_eval(rt, s.rdeg, xa, &psi, &dpsi);
      const R Fhat = sc.A * psi / k2;
      const R dterm = sc.A * xa * dpsi / (k2 * k2);
      const R a = (X.x * X.x + X.y * X.y) * iw * sc.scale;
      const R aF = a * Fhat;
      const R ckk = a * (dterm - R(2) * Fhat / k2);
      const R contrib[7] = {aF,
                            aF + ckk * kx * kx,
                            aF + ckk * ky * ky,
                            aF + ckk * kz * kz,
                            ckk * kx * ky,
                            ckk * kx * kz,
                            ckk * ky * kz};
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        if constexpr (kD)
          acc[j] += contrib[j];
        else
          acc[j].add(contrib[j]);
      }
      if (INV) {
        // conjugated: the inverse transform is the forward one between two conjugations
        const R G = Fhat * iw0[i0] * cg[c];
        cur[e] = cmk<R>(X.x * G, -X.y * G);
      }
    }
    if (INV) {
      __syncthreads();
      cur = xfft_lines<R, -1>(cur, oth, tw, x);
      for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int c = e & (NC - 1), f = f0 + c;
        if (f < x.ncol) {
          C v = cur[e];
          v.y = -v.y;
          out[(int64_t)(e >> lognc) * rowst + f] = v;
        }
      }
    }
  }
  {
    // the CTA's sums in a fixed order (FP32: compensated pairs); k_xsum adds them up
    __shared__ Acc red[7][kXThreads / 32];
    const Acc t = cta_sum7<Acc, kXThreads / 32>(acc, red);
    if (threadIdx.x < 7) {
      if constexpr (kD)
        partials[(size_t)threadIdx.x * nactive + blockIdx.x] = t;
      else
        reinterpret_cast<float2*>(partials)[(size_t)threadIdx.x * nactive + blockIdx.x] =
            make_float2(t.hi, t.lo);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Plane transforms over (i1, i2), one CTA per plane i0, pruned to the box of the sphere
// |m1| <= mmax1, 0 <= m2 <= mmax2 (every mode with |k| <= c / r_c lies in it).  Shared
// memory (complex elements): the M1 and M2 roots, T = M1 x ncb (the lines along i1, one
// column per m2) and a work area of max(2 M2 nca, M1 ncb).
template <typename R>
__host__ __device__ constexpr int plane_threads() {
  return std::is_same<R, float>::value ? 2 * kPThreads : kPThreads;
}

__host__ __device__ inline size_t plane_smem_elems(const PlaneGeom& pg) {
  const size_t t = (size_t)pg.M1 * pg.b.nc;
  const size_t w1 = 2 * (size_t)pg.M2 * pg.a.nc;
  return (size_t)pg.M1 + pg.M2 + t + (w1 > t ? w1 : t);
}

// Forward: the real lines along i2 are taken two at a time as one complex line z = x_a +
// i x_b; from its transform Z, X_a(m) = (Z(m) + conj Z(-m)) / 2 and X_b(m) = (Z(m) - conj
// Z(-m)) / (2 i) for m2 = m < nb2.  Then the transform along i1 of those nb2 columns, of
// which the nb1 rows of the box are written to box[i0][b1][m2].
template <typename R>
__global__ void __launch_bounds__(plane_threads<R>()) k_fplane(const R* __restrict__ grid,
                                                      typename Cplx<R>::T* __restrict__ box,
                                                      PlaneGeom pg,
                                                      const typename Cplx<R>::T* __restrict__ twg) {
  pdl_wait();
  using C = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M1 = pg.M1, M2 = pg.M2, nca = pg.a.nc, ncb = pg.b.nc, nb2 = pg.nb2;
  C* twB = reinterpret_cast<C*>(smem_raw);
  C* twA = twB + M1;
  C* T = twA + M2;
  C* U = T + (size_t)M1 * ncb;
  C* U2 = U + (size_t)M2 * nca;
  for (int e = threadIdx.x; e < M1 + M2; e += blockDim.x) twB[e] = twg[e];
  const R* plane = grid + (size_t)blockIdx.x * M1 * M2;
  for (int p0 = 0; p0 < pg.npairs; p0 += pg.pairs_b) {
    const int np = min(pg.pairs_b, pg.npairs - p0);
    __syncthreads();  // the work area is free, the roots are in place
    // kU elements per thread and round, all loads issued before the first store
    constexpr int kU = 8;
    for (int e0 = threadIdx.x; e0 < M2 * nca; e0 += kU * blockDim.x) {
      R re[kU], im[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = e0 + u * blockDim.x;
        const int c = fast_div(e, pg.m2_magic);
        const int j = e - c * M2;
        const int r = 2 * (p0 + c);
        re[u] = (e < M2 * nca && c < np) ? plane[(size_t)r * M2 + j] : R(0);
        im[u] = (e < M2 * nca && c < np && r + 1 < M1) ? plane[(size_t)(r + 1) * M2 + j] : R(0);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < M2 * nca) {
          const int c = fast_div(e, pg.m2_magic);
          const int j = e - c * M2;
          U[j * nca + c] = cmk<R>(re[u], im[u]);
        }
      }
    }
    __syncthreads();
    const C* Z = lfft_any<R, -1>(U, U2, twA, pg.a);
    for (int e = threadIdx.x; e < nb2 * np; e += blockDim.x) {
      const int c = fast_div(e, pg.nb2_magic);
      const int m = e - c * nb2;
      const C z = Z[m * nca + c];
      const C w = Z[(m == 0 ? 0 : M2 - m) * nca + c];
      const int r = 2 * (p0 + c);
      T[r * ncb + m] = cmk<R>(R(0.5) * (z.x + w.x), R(0.5) * (z.y - w.y));
      if (r + 1 < M1) T[(r + 1) * ncb + m] = cmk<R>(R(0.5) * (z.y + w.y), R(0.5) * (w.x - z.x));
    }
  }
  __syncthreads();
  const C* Y = lfft_any<R, -1>(T, U, twB, pg.b);
  C* out = box + (size_t)blockIdx.x * pg.nb1 * nb2;
  for (int e = threadIdx.x; e < pg.nb1 * nb2; e += blockDim.x) {
    const int b1 = fast_div(e, pg.nb2_magic);
    const int m = e - b1 * nb2;
    const int m1 = (2 * b1 <= pg.nb1) ? b1 : b1 - pg.nb1;
    out[e] = Y[(m1 < 0 ? m1 + M1 : m1) * ncb + m];
  }
}

// Inverse (unnormalised, as the forward): the box columns (zero where colact = 0 and
// outside the box) take the inverse transform along i1, then pairs of lines along i2 are
// rebuilt as Z(m) = X_a(m) + i X_b(m) over the Hermitian extension X(-m) = conj X(m) (the
// m = 0 term real) and transformed, x_a = Re, x_b = Im.  Inverse transforms are forward
// ones between two conjugations.
template <typename R, typename G>
__global__ void __launch_bounds__(plane_threads<R>()) k_iplane(const typename Cplx<R>::T* __restrict__ box,
                                                      const unsigned char* __restrict__ colact,
                                                      G* __restrict__ grid, PlaneGeom pg,
                                                      const typename Cplx<R>::T* __restrict__ twg) {
  pdl_wait();
  using C = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M1 = pg.M1, M2 = pg.M2, nca = pg.a.nc, ncb = pg.b.nc, nb2 = pg.nb2;
  C* twB = reinterpret_cast<C*>(smem_raw);
  C* twA = twB + M1;
  C* T = twA + M2;
  C* U = T + (size_t)M1 * ncb;
  C* U2 = U + (size_t)M2 * nca;
  for (int e = threadIdx.x; e < M1 + M2; e += blockDim.x) twB[e] = twg[e];
  for (int e = threadIdx.x; e < M1 * ncb; e += blockDim.x) T[e] = cmk<R>(R(0), R(0));
  __syncthreads();
  const C* in = box + (size_t)blockIdx.x * pg.nb1 * nb2;
  {
    // the box columns, kU per thread and round with every load issued first (the
    // inactive columns hold stale values and are replaced by zero)
    constexpr int kU = 4;
    const int nbox = pg.nb1 * nb2;
    for (int e0 = threadIdx.x; e0 < nbox; e0 += kU * blockDim.x) {
      C v[kU];
      unsigned char a[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = e0 + u * blockDim.x;
        a[u] = e < nbox ? colact[e] : 0;
        v[u] = e < nbox ? in[e] : cmk<R>(R(0), R(0));
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < nbox) {
          const int b1 = fast_div(e, pg.nb2_magic);
          const int m = e - b1 * nb2;
          const int m1 = (2 * b1 <= pg.nb1) ? b1 : b1 - pg.nb1;
          T[(m1 < 0 ? m1 + M1 : m1) * ncb + m] = a[u] ? cmk<R>(v[u].x, -v[u].y) : cmk<R>(R(0), R(0));
        }
      }
    }
  }
  __syncthreads();
  C* Yc = lfft_any<R, -1>(T, U, twB, pg.b);  // conj of the inverse along i1
  if (Yc != T) {
    for (int e = threadIdx.x; e < M1 * ncb; e += blockDim.x) T[e] = Yc[e];
  }
  G* plane = grid + (size_t)blockIdx.x * M1 * M2;
  for (int p0 = 0; p0 < pg.npairs; p0 += pg.pairs_b) {
    const int np = min(pg.pairs_b, pg.npairs - p0);
    __syncthreads();  // T complete; the work area is free
    for (int e = threadIdx.x; e < M2 * nca; e += blockDim.x) {
      const int c = fast_div(e, pg.m2_magic);
      const int j = e - c * M2;
      C z = cmk<R>(R(0), R(0));
      if (c < np) {
        const int r = 2 * (p0 + c);
        const bool two = r + 1 < M1;
        if (j < nb2) {
          // a = X_a(j), b = X_b(j) (T holds their conjugates)
          const C ta = T[r * ncb + j];
          const C tb = two ? T[(r + 1) * ncb + j] : cmk<R>(R(0), R(0));
          z = j == 0 ? cmk<R>(ta.x, tb.x) : cmk<R>(ta.x + tb.y, tb.x - ta.y);
        } else if (j > M2 - nb2) {
          // conj X_a(M2 - j) + i conj X_b(M2 - j)
          const int m = M2 - j;
          const C ta = T[r * ncb + m];
          const C tb = two ? T[(r + 1) * ncb + m] : cmk<R>(R(0), R(0));
          z = cmk<R>(ta.x - tb.y, ta.y + tb.x);
        }
      }
      z.y = -z.y;
      U[j * nca + c] = z;
    }
    __syncthreads();
    const C* Zc = lfft_any<R, -1>(U, U2, twA, pg.a);  // conj of the inverse along i2
    for (int e = threadIdx.x; e < M2 * np; e += blockDim.x) {
      const int c = fast_div(e, pg.m2_magic);
      const int j = e - c * M2;
      const C v = Zc[j * nca + c];
      const int r = 2 * (p0 + c);
      plane[(size_t)r * M2 + j] = grid_elem<G>(v.x);
      if (r + 1 < M1) plane[(size_t)(r + 1) * M2 + j] = grid_elem<G>(-v.y);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Force gather.  Persistent CTAs take tiles from a global counter (ctrl[5]) two ahead of
// the one they work on, and copy the next tile's padded block of the potential grid, its
// atom count and its first chunk of atoms into the other half of a double buffer with
// asynchronous copies while the current tile is worked on.  Per chunk of a tile's atoms:
// (A) thread (p, a) evaluates the window and its derivative at stencil point p for the
// three dimensions of atom a (three packed Horner chains); (B) groups of P lanes take one
// atom each (32 / P atoms per warp at a time): lane j of a group contracts stencil row j
// (its P x P points) in registers, a segmented shuffle reduction sums the rows, and the
// group's first lane turns the sums into the atom's force.
template <typename R, typename IO, int P, typename G>
__global__ void __launch_bounds__(kThreads, std::is_same<R, float>::value ? 3 : 2) k_gather(
    Bins bins, GatherGeom gg, int ntiles, const R* __restrict__ wtab,
    const G* __restrict__ grid, IO* __restrict__ forces) {
  pdl_wait();
  const TileGeom& g = gg.g;
  using V4 = typename Vec4<R>::T;
  constexpr int ES = (int)sizeof(R);
  constexpr int GS = (int)sizeof(G);  // potential grid element: the compute type or BF16
  constexpr int CH = gather_chunk(ES);
  constexpr int PS = round_up4(P), RS = record_stride(true, P);
  constexpr int T2c = P <= 8 ? 16 : 8;
  constexpr int E1 = 8 + P - 1, E3 = gather_pitch(T2c + P - 1, GS), S1 = E1 * E3;
  constexpr int VOL = (8 + P - 1) * S1;
  constexpr int VW = 16 / GS;  // elements per 16-byte copy
  const GatherLayout L = gather_layout(ES, P, GS);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  G* phi_b = reinterpret_cast<G*>(smem_raw + L.phi);  // 2 x VOL
  R* W = reinterpret_cast<R*>(smem_raw + L.w);        // per atom [w0|w1|w2|w0'|w1'|w2']
  V4* TQ_b = reinterpret_cast<V4*>(smem_raw + L.tq);  // 2 x CH
  int* LB_b = reinterpret_cast<int*>(smem_raw + L.lb);
  int* X_b = reinterpret_cast<int*>(smem_raw + L.idx);
  int* CNT_b = reinterpret_cast<int*>(smem_raw + L.cnt);
  const V4* __restrict__ slot_tq = static_cast<const V4*>(bins.tq);
  // tiles taken ahead, with the grid origin of each (computed once, by the thread that
  // takes the tile)
  __shared__ int s_first[2], s_ahead[2];
  __shared__ int3 s_ofirst[2], s_oahead[2];

  constexpr int D = WinDeg<R>::value;
  constexpr int NPA = kThreads / P;  // atoms per sweep of the window evaluation
  constexpr int GA = 32 / P;         // atoms per warp at a time
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = lane / P, jj = lane - slot * P;
  const int p_t = threadIdx.x % P, a_t = threadIdx.x / P;
  const int E0 = g.E[0], E1r = g.E[1], E2 = g.E[2];
  const int ncopy = min(CH, bins.cap);

  // thread 0 takes a tile and records its grid origin
  auto take = [&](int* st, int3* so) {
    const int t = atomicAdd(&bins.ctrl[5], 1);
    *st = t;
    if (t < ntiles) {
      const int t2 = t % g.nt[2];
      const int t1 = (t / g.nt[2]) % g.nt[1];
      const int t0 = t / (g.nt[2] * g.nt[1]);
      *so = make_int3(t0 * g.T[0], t1 * g.T[1], t2 * g.T[2]);
    }
  };
  // copies of tile t (origin o) into buffer b: block, count, first chunk of atoms (one group)
  auto issue = [&](int t, int3 o, int b) {
    if (t < ntiles) {
      const int o0 = o.x, o1 = o.y, o2 = o.z;
      G* phi = phi_b + b * VOL;
      if (g.gvec) {
        const int E2v = g.E2g;
        const int n = E0 * E1r * E2v;
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
          const int ab = fast_div(e, g.div_E2g), c4 = e - ab * E2v;
          const int a = fast_div(ab, g.div_E1), bb = ab - a * E1r;
          const int gi = wrap3(o0 + a, g.M[0]);
          const int gj = wrap3(o1 + bb, g.M[1]);
          const int gk = wrap3(o2 + VW * c4, g.M[2]);
          cp_async16(phi + a * S1 + bb * E3 + VW * c4,
                     grid + ((int64_t)gi * g.M[1] + gj) * g.M[2] + gk);
        }
      } else if constexpr (GS >= 4) {
        // (a BF16 grid always takes the 16-byte path: the plan requires it)
        const int n = E0 * E1r * E2;
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
          const int ab = e / E2, c = e - ab * E2;
          const int a = ab / E1r, bb = ab - a * E1r;
          const int gi = wrap_index(o0 + a, g.M[0]);
          const int gj = wrap_index(o1 + bb, g.M[1]);
          const int gk = wrap_index(o2 + c, g.M[2]);
          cp_async_small<GS>(phi + a * S1 + bb * E3 + c,
                             grid + ((int64_t)gi * g.M[1] + gj) * g.M[2] + gk);
        }
      }
      // atoms: the slot arrays are padded by a chunk, so whole chunks stay in bounds
      const int64_t s0 = (int64_t)t * bins.cap;
      constexpr int QV = (int)sizeof(V4) / 16;  // 16-byte pieces per (t, q) record
      for (int e = threadIdx.x; e < ncopy * QV; e += blockDim.x)
        cp_async16(reinterpret_cast<unsigned char*>(TQ_b + b * CH) + 16 * e,
                   reinterpret_cast<const unsigned char*>(slot_tq + s0) + 16 * e);
      const int ni = (ncopy + 3) / 4;
      for (int e = threadIdx.x; e < 2 * ni; e += blockDim.x) {
        if (e < ni)
          cp_async16(LB_b + b * CH + 4 * e, bins.lb + s0 + 4 * e);
        else
          cp_async16(X_b + b * CH + 4 * (e - ni), bins.idx + s0 + 4 * (e - ni));
      }
      if (threadIdx.x == 0) cp_async_small<4>(CNT_b + b, bins.tcount + t);
    }
    cp_async_commit();
  };

  if (threadIdx.x == 0) {
    take(&s_first[0], &s_ofirst[0]);
    take(&s_first[1], &s_ofirst[1]);
  }
  __syncthreads();
  int cur = s_first[0], nxt = s_first[1];
  issue(cur, s_ofirst[0], 0);
  issue(nxt, s_ofirst[1], 1);

  for (int k = 0; cur < ntiles; ++k) {
    const int b = k & 1;
    if (threadIdx.x == 0) take(&s_ahead[b], &s_oahead[b]);
    cp_async_wait<1>();
    __syncthreads();  // tile cur's block and atoms are in buffer b
    const G* phi = phi_b + b * VOL;
    V4* TQ = TQ_b + b * CH;
    int* LB = LB_b + b * CH;
    int* X = X_b + b * CH;
    const int cnt_all = CNT_b[b];
    const int64_t s0 = (int64_t)cur * bins.cap;
    for (int c0 = 0; c0 < cnt_all; c0 += CH) {
      const int cnt = min(CH, cnt_all - c0);
      if (c0 > 0) {
        // a tile with more atoms than a chunk: the later chunks are loaded here
        __syncthreads();
        for (int a = threadIdx.x; a < cnt; a += blockDim.x) {
          TQ[a] = slot_tq[s0 + c0 + a];
          LB[a] = bins.lb[s0 + c0 + a];
          X[a] = bins.idx[s0 + c0 + a];
        }
        __syncthreads();
      }
      // (A) window values and derivatives: thread (p_t, a) for the three dimensions
      if (a_t < NPA) {
        if constexpr (std::is_same<R, float>::value) {
          unsigned long long cwd[D + 1];
#pragma unroll
          for (int kk = 0; kk <= D; ++kk)
            cwd[kk] = pack2(__ldg(wtab + kk * P + p_t), __ldg(wtab + (D + 1) * P + kk * P + p_t));
          for (int a = a_t; a < cnt; a += NPA) {
            const V4 v = TQ[a];
            float w0, d0, w1, d1, w2, d2;
            unpack2(horner2<D>(cwd, pack2(v.x - 0.5f, v.x - 0.5f)), w0, d0);
            unpack2(horner2<D>(cwd, pack2(v.y - 0.5f, v.y - 0.5f)), w1, d1);
            unpack2(horner2<D>(cwd, pack2(v.z - 0.5f, v.z - 0.5f)), w2, d2);
            R* Wa = W + a * RS + p_t;
            Wa[0] = w0;
            Wa[PS] = w1;
            Wa[2 * PS] = w2;
            Wa[3 * PS] = d0 * g.dscalef[0];
            Wa[4 * PS] = d1 * g.dscalef[1];
            Wa[5 * PS] = d2 * g.dscalef[2];
          }
        } else {
          R cw[D + 1], cd[D + 1];
#pragma unroll
          for (int kk = 0; kk <= D; ++kk) {
            cw[kk] = __ldg(wtab + kk * P + p_t);
            cd[kk] = __ldg(wtab + (D + 1) * P + kk * P + p_t);
          }
          for (int a = a_t; a < cnt; a += NPA) {
            const V4 v = TQ[a];
            R* Wa = W + a * RS + p_t;
            Wa[0] = horner_reg<R, D>(cw, v.x);
            Wa[PS] = horner_reg<R, D>(cw, v.y);
            Wa[2 * PS] = horner_reg<R, D>(cw, v.z);
            Wa[3 * PS] = horner_reg<R, D>(cd, v.x) * g.dscale[0];
            Wa[4 * PS] = horner_reg<R, D>(cd, v.y) * g.dscale[1];
            Wa[5 * PS] = horner_reg<R, D>(cd, v.z) * g.dscale[2];
          }
        }
      }
      __syncthreads();
      // (B) lane j of an atom's group: the P x P points (i, k) of row j in registers
      //   gx = w1[j] sum_k w2[k] sum_i phi w0'[i],  gy = w1'[j] sum_k w2[k] sum_i phi w0[i],
      //   gz = w1[j] sum_k w2'[k] sum_i phi w0[i]
      for (int a0 = warp * GA; a0 < cnt; a0 += (kThreads / 32) * GA) {
        const int a = a0 + slot;
        const bool valid = slot < GA && a < cnt;
        R ax = R(0), ay = R(0), az = R(0);
        if (valid) {
          const R* Wa = W + a * RS;
          R w0[P], d0[P], w2[P], d2[P];
          load_record<R, P>(Wa, w0);
          load_record<R, P>(Wa + 2 * PS, w2);
          load_record<R, P>(Wa + 3 * PS, d0);
          load_record<R, P>(Wa + 5 * PS, d2);
          const int lb = LB[a];
          const G* src = phi + (lb & 1023) * S1 + (((lb >> 10) & 1023) + jj) * E3 + ((lb >> 20) & 1023);
#pragma unroll
          for (int kk = 0; kk < P; ++kk) {
            R sx = R(0), sw = R(0);
#pragma unroll
            for (int i = 0; i < P; ++i) {
              const R f = grid_val(src[i * S1 + kk]);
              sx = fma(f, d0[i], sx);
              sw = fma(f, w0[i], sw);
            }
            ax = fma(w2[kk], sx, ax);
            ay = fma(w2[kk], sw, ay);
            az = fma(d2[kk], sw, az);
          }
          const R w1 = Wa[PS + jj];
          ax *= w1;
          ay *= Wa[4 * PS + jj];
          az *= w1;
        }
        // segmented sum: lane j of a group ends with rows j .. P-1 of its atom
#pragma unroll
        for (int sft = 1; sft < P; sft <<= 1) {
          const R tx = __shfl_down_sync(0xffffffffu, ax, sft);
          const R ty = __shfl_down_sync(0xffffffffu, ay, sft);
          const R tz = __shfl_down_sync(0xffffffffu, az, sft);
          if (jj + sft < P) {
            ax += tx;
            ay += ty;
            az += tz;
          }
        }
        if (valid && jj == 0) {
          // dU/ds = -(q / (V Mtot^2)) (gx, gy, gz);  F = -h^{-T} dU/ds
          const int idx = X[a];
          const R qa = TQ[a].w;
          if constexpr (std::is_same<R, float>::value) {
            const float f = qa * gg.fscalef;
#pragma unroll
            for (int c = 0; c < 3; ++c)
              forces[3 * (int64_t)idx + c] =
                  (IO)(f * (g.hinvf[c] * ax + g.hinvf[3 + c] * ay + g.hinvf[6 + c] * az));
          } else {
            const double f = qa * gg.fscale;
#pragma unroll
            for (int c = 0; c < 3; ++c)
              forces[3 * (int64_t)idx + c] =
                  (IO)(f * (g.hinv[c] * ax + g.hinv[3 + c] * ay + g.hinv[6 + c] * az));
          }
        }
      }
    }
    __syncthreads();  // buffer b is free; s_ahead[b] is visible
    const int nn = s_ahead[b];
    const int3 nn_o = s_oahead[b];
    issue(nn, nn_o, b);
    cur = nxt;
    nxt = nn;
  }
  cp_async_wait<0>();
  __syncthreads();

  // atoms past their tile's capacity: one warp per atom, straight from the global grid
  {
    const int novf = bins.ctrl[4];
    R* Ww = W + warp * (6 * kMaxP);
    const typename Vec4<R>::T* otq = static_cast<const typename Vec4<R>::T*>(bins.otq);
    for (;;) {
      int o = 0;
      if (lane == 0) o = atomicAdd(&bins.ctrl[6], 1);
      o = __shfl_sync(0xffffffffu, o, 0);
      if (o >= novf) break;
      const typename Vec4<R>::T v = otq[o];
      const int b0 = bins.ob[3 * o], b1 = bins.ob[3 * o + 1], b2 = bins.ob[3 * o + 2];
      for (int e = lane; e < 3 * P; e += 32) {
        const int d = e / P, pp = e - d * P;
        const R tau = tq_comp<R>(v, d) - R(0.5);
        R w = wtab[D * P + pp], dw = wtab[(D + 1) * P + D * P + pp];
        for (int k = D - 1; k >= 0; --k) {
          w = fma(w, tau, wtab[k * P + pp]);
          dw = fma(dw, tau, wtab[(D + 1) * P + k * P + pp]);
        }
        Ww[e] = w;
        Ww[3 * P + e] = dw * dscale_of<R>(g, d);
      }
      __syncwarp();
      R ax = R(0), ay = R(0), az = R(0);
      for (int l = lane; l < P * P * P; l += 32) {
        const int i = l / (P * P), r = l - i * (P * P), j = r / P, k = r - j * P;
        const int gi = wrap_index(b0 + i, g.M[0]);
        const int gj = wrap_index(b1 + j, g.M[1]);
        const int gk = wrap_index(b2 + k, g.M[2]);
        const R f = grid_val(grid[((int64_t)gi * g.M[1] + gj) * g.M[2] + gk]);
        ax = fma(f, Ww[3 * P + i] * Ww[P + j] * Ww[2 * P + k], ax);
        ay = fma(f, Ww[i] * Ww[4 * P + j] * Ww[2 * P + k], ay);
        az = fma(f, Ww[i] * Ww[P + j] * Ww[5 * P + k], az);
      }
#pragma unroll
      for (int sft = 16; sft > 0; sft >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, sft);
        ay += __shfl_xor_sync(0xffffffffu, ay, sft);
        az += __shfl_xor_sync(0xffffffffu, az, sft);
      }
      if (lane == 0) {
        const int idx = bins.oidx[o];
        const double f = (double)v.w * gg.fscale;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          forces[3 * (int64_t)idx + c] =
              (IO)(f * (g.hinv[c] * (double)ax + g.hinv[3 + c] * (double)ay + g.hinv[6 + c] * (double)az));
      }
      __syncwarp();
    }
  }
  last_cta_resets(bins.ctrl, 7, 5, 3);
}

// ---------------------------------------------------------------------------------------
// Cell gradient of the long-range energy at fixed Cartesian positions (Sec. 2.2, eq.
// (instheta) with r = h s): dU/dh = -W h^{-T} + sum_i F_i s_i^T, s_i = h^{-1} r_i as given
// (unwrapped), W = W_F + U_bg I.  grad (row-major, zeroed by the host) receives each
// block's part of the moment sum; block 0 adds -W h^{-T} from the step's accumulator.
template <typename IO>
__global__ void __launch_bounds__(kThreads) k_cell_grad(const IO* __restrict__ pos,
                                                        const IO* __restrict__ F, int64_t n,
                                                        CellGradArgs c,
                                                        const double* __restrict__ acc,
                                                        double* __restrict__ grad) {
  double m[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) m[e] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double r[3] = {(double)pos[3 * i], (double)pos[3 * i + 1], (double)pos[3 * i + 2]};
    if (!(isfinite(r[0]) && isfinite(r[1]) && isfinite(r[2]))) continue;  // skipped atoms
    const double f[3] = {(double)F[3 * i], (double)F[3 * i + 1], (double)F[3 * i + 2]};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const double sb = c.hinv[3 * b] * r[0] + c.hinv[3 * b + 1] * r[1] + c.hinv[3 * b + 2] * r[2];
#pragma unroll
      for (int a = 0; a < 3; ++a) m[3 * a + b] += f[a] * sb;
    }
  }
  __shared__ double part[kThreads / 32][9];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const double v = warp_sum(m[e]);
    if (lane == 0) part[warp][e] = v;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) v += part[w][threadIdx.x];
    if (blockIdx.x == 0) {
      // -(W h^{-T})_{ab} = -sum_c W_ac hinv_bc, W = W_F + U_bg I (accumulator: xx yy zz xy xz yz)
      const double ubg = c.bg_coef * acc[7] * acc[7];
      const double W[9] = {acc[1] + ubg, acc[4], acc[5], acc[4], acc[2] + ubg, acc[6],
                           acc[5], acc[6], acc[3] + ubg};
      const int a = threadIdx.x / 3, b = threadIdx.x % 3;
      v -= W[3 * a] * c.hinv[3 * b] + W[3 * a + 1] * c.hinv[3 * b + 1] + W[3 * a + 2] * c.hinv[3 * b + 2];
    }
    atomicAdd(grad + threadIdx.x, v);
  }
}

// ---------------------------------------------------------------------------------------
// Near part of the split (Sec. 3, eqs. (UN), (Fc), (PinsN) with the sign of -dU/dh h^T):
// U_N = 1/2 sum' q_i q_j N(r), N(r) = (1 - phi_0(r/r_c)) / r on r <= r_c; the force on i
// sum_j q_i q_j F_N(r) r_ij / r^3 with F_N = 1 - phi_0 + u psi_0(u) / C_0; the virial
// 1/2 sum' q_i q_j F_N(r) r_ij (x) r_ij / r^3.  Both functions of u = r / r_c come from
// piecewise polynomials (the radial table layout).

// FP32 sums compensated, FP64 sums plain
template <typename R>
struct Sum;
template <>
struct Sum<float> {
  DF d;
  __device__ __forceinline__ void add(float v) { d.add(v); }
  __device__ __forceinline__ double value() const { return (double)d.hi + (double)d.lo; }
};
template <>
struct Sum<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ double value() const { return v; }
};

template <typename IO, typename R>
__global__ void __launch_bounds__(kThreads) k_near_bin(const IO* __restrict__ pos,
                                                       const IO* __restrict__ q, int64_t n,
                                                       NearGeom ng, int* __restrict__ ccount,
                                                       int* __restrict__ cell,
                                                       int* __restrict__ rank,
                                                       typename Vec4<R>::T* __restrict__ xq) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double r[3] = {(double)pos[3 * i], (double)pos[3 * i + 1], (double)pos[3 * i + 2]};
    const double qi = (double)q[i];
    if (!(isfinite(r[0]) && isfinite(r[1]) && isfinite(r[2]) && isfinite(qi))) {
      cell[i] = -1;
      continue;
    }
    int c[3];
    double f[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double sd = ng.hinv[3 * d] * r[0] + ng.hinv[3 * d + 1] * r[1] + ng.hinv[3 * d + 2] * r[2];
      sd -= floor(sd);
      if (sd >= 1.0) sd = 0.0;
      const double td = sd * ng.nc[d];
      c[d] = min((int)td, ng.nc[d] - 1);
      f[d] = (td - (double)c[d]) * ng.inv_nc[d];  // reduced offset from the cell corner
    }
    const int id = (c[0] * ng.nc[1] + c[1]) * ng.nc[2] + c[2];
    cell[i] = id;
    rank[i] = atomicAdd(&ccount[id], 1);
    typename Vec4<R>::T v;
    v.x = (R)(ng.h[0] * f[0] + ng.h[1] * f[1] + ng.h[2] * f[2]);
    v.y = (R)(ng.h[3] * f[0] + ng.h[4] * f[1] + ng.h[5] * f[2]);
    v.z = (R)(ng.h[6] * f[0] + ng.h[7] * f[1] + ng.h[8] * f[2]);
    v.w = (R)qi;
    xq[i] = v;
  }
}

// Exclusive scan of the cell counts by one CTA of kScanThreads threads, kScanPer counts
// per thread and pass; ccount is zeroed for the next call.
constexpr int kScanThreads = 1024, kScanPer = 8;
__global__ void __launch_bounds__(kScanThreads) k_near_scan(int* __restrict__ ccount,
                                                            int* __restrict__ coff, int ncells) {
  __shared__ int wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int carry = 0;
  for (int base = 0; base < ncells; base += kScanPer * kScanThreads) {
    int v[kScanPer], sum = 0;
    const int i0 = base + kScanPer * threadIdx.x;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      v[k] = i0 + k < ncells ? ccount[i0 + k] : 0;
      sum += v[k];
    }
#pragma unroll
    for (int k = 0; k < kScanPer; ++k)
      if (i0 + k < ncells) ccount[i0 + k] = 0;
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int t = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      wsum[lane] = t;
    }
    __syncthreads();
    int o = carry + (wid > 0 ? wsum[wid - 1] : 0) + x - sum;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
      if (i0 + k < ncells) coff[i0 + k] = o;
      o += v[k];
    }
    carry += wsum[kScanThreads / 32 - 1];
    __syncthreads();  // wsum is reused
  }
  if (threadIdx.x == 0) coff[ncells] = carry;
}

template <typename V>
__global__ void __launch_bounds__(kThreads) k_near_scatter(int64_t n, const int* __restrict__ cell,
                                                           const int* __restrict__ rank,
                                                           const int* __restrict__ coff,
                                                           V* __restrict__ xq_tmp,
                                                           V* __restrict__ xq,
                                                           int* __restrict__ idx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = cell[i];
    if (c >= 0) {
      const int dst = coff[c] + rank[i];
      xq[dst] = xq_tmp[i];
      idx[dst] = (int)i;
    }
    // the array is the pair kernel's force accumulator next
    memset(static_cast<void*>(xq_tmp + i), 0, sizeof(V));
  }
}

// sum over the warp of a compensated FP32 value (or a double on the FP64 path)
__device__ __forceinline__ double warp_total(const Sum<float>& s) {
  DF v = s.d;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v.add(w);
  }
  return (double)v.hi + (double)v.lo;
}
__device__ __forceinline__ double warp_total(const Sum<double>& s) { return warp_sum(s.v); }

// Candidates (atoms of the block's neighbourhood) a CTA holds in shared memory at a time.
template <typename R>
__host__ __device__ constexpr int near_cand() {
  return std::is_same<R, float>::value ? 1536 : 1024;
}
// dynamic shared memory of k_near_pairs for a neighbourhood of nreg cells and nh x nrow
// home-cell rows: candidates (position, charge) and their force sums (3 per candidate),
// per cell its displacement, first sorted index and the prefix sum of the atom counts,
// and the row ranges
__host__ __device__ inline size_t near_smem_bytes(bool fp64, int nreg, int nrows) {
  const size_t es = fp64 ? 8 : 4;
  const size_t kc = fp64 ? near_cand<double>() : near_cand<float>();
  return kc * (4 * es + 3 * es) + (size_t)nreg * (4 * es + 2 * sizeof(int)) +
         2 * sizeof(int) + (size_t)nrows * 2 * sizeof(int);
}

// psi pair of the near kernel: N-part factor g1 = 1 - phi_0(u) and force factor
// g2 = 1 - phi_0(u) + u psi_0(u) / C_0 from a shared-memory table of kRadialPieces pieces
// with interleaved coefficients (g1_k, g2_k) of (u - centre)^k, degree ND (compile time)
// or nd (ND = 0).  FP32: both polynomials in step as packed pairs.
template <int ND>
__device__ __forceinline__ void near_eval(const float2* __restrict__ t2, int nd, float u,
                                          float* g1, float* g2) {
  if constexpr (ND > 0) nd = ND;
  int piece = (int)(u * (float)kRadialPieces);
  piece = piece < 0 ? 0 : (piece >= kRadialPieces ? kRadialPieces - 1 : piece);
  const float tau = u - ((float)piece + 0.5f) / (float)kRadialPieces;
  const unsigned long long* c = reinterpret_cast<const unsigned long long*>(t2 + piece * (nd + 1));
  const unsigned long long tt = pack2(tau, tau);
  unsigned long long v = c[nd];
  if constexpr (ND > 0) {
#pragma unroll
    for (int k = ND - 1; k >= 0; --k) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(v) : "l"(tt), "l"(c[k]));
  } else {
    for (int k = nd - 1; k >= 0; --k) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(v) : "l"(tt), "l"(c[k]));
  }
  unpack2(v, *g1, *g2);
}
template <int ND>
__device__ __forceinline__ void near_eval(const double2* __restrict__ t2, int nd, double u,
                                          double* g1, double* g2) {
  if constexpr (ND > 0) nd = ND;
  int piece = (int)(u * (double)kRadialPieces);
  piece = piece < 0 ? 0 : (piece >= kRadialPieces ? kRadialPieces - 1 : piece);
  const double tau = u - ((double)piece + 0.5) / (double)kRadialPieces;
  const double2* c = t2 + piece * (nd + 1);
  double a = c[nd].x, b = c[nd].y;
  for (int k = nd - 1; k >= 0; --k) {
    a = fma(a, tau, c[k].x);
    b = fma(b, tau, c[k].y);
  }
  *g1 = a;
  *g2 = b;
}

// Displacements of a block's neighbourhood cells: entry ((r0 Y) + r1) Z + r2 of the
// largest neighbourhood (Y = B1 + 2 R1, Z = B2 + 2 R2) is h (r0, r1 - R1, r2 - R2) / nc,
// the corner of that cell relative to the block's corner cell.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_near_offsets(NearGeom ng,
                                                           typename Vec4<R>::T* __restrict__ off) {
  const int Y = ng.B[1] + 2 * ng.R[1], Z = ng.B[2] + 2 * ng.R[2];
  const int n = (ng.B[0] + ng.R[0]) * Y * Z;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int r0 = t / (Y * Z), r1 = (t / Z) % Y - ng.R[1], r2 = t % Z - ng.R[2];
    const double f0 = (double)r0 / ng.nc[0], f1 = (double)r1 / ng.nc[1], f2 = (double)r2 / ng.nc[2];
    typename Vec4<R>::T d;
    d.x = (R)(ng.h[0] * f0 + ng.h[1] * f1 + ng.h[2] * f2);
    d.y = (R)(ng.h[3] * f0 + ng.h[4] * f1 + ng.h[5] * f2);
    d.z = (R)(ng.h[6] * f0 + ng.h[7] * f1 + ng.h[8] * f2);
    d.w = R(0);
    off[t] = d;
  }
}

// Half-shell pair sum of the near part.  A CTA takes a block of B0 x B1 x B2 cells of the
// cell list (cells at least r_c / 2 wide, reach R cells per side).  Each pair of atoms and
// periodic image is met once: from the cell c of atom i, the offsets o in [-R, R]^3 that
// come after (0, 0, 0) in the order (o0, o1, o2), and within c itself the atoms after i.
// The CTA's neighbourhood is the (hb0 + R0) x (hb1 + 2 R1) x (hb2 + 2 R2) cells that these
// offsets reach from its block, held in shared memory as rows along axis 2 (a row of
// consecutive cells is one contiguous range of candidates), positions relative to the
// block's corner cell.  A warp takes one atom of the block at a time; its lanes stride
// over the 2 R2 + 1 cells of each forward row, and the pairs within r_c go through a warp
// queue of candidate slots (ballot and population count) and are worked 32 at a time.  The pair force goes
// to atom i in registers (summed over the warp once per atom) and, with the opposite
// sign, to the candidate's sums in shared memory; those are added once per chunk to the
// sorted-order accumulator fsort (vector atomics).  Energy and virial count each pair
// once; the FP32 path sums them per lane in plain precision over a chunk and adds that to
// compensated running sums.
template <typename R, int ND>
__global__ void __launch_bounds__(kThreads, 4) k_near_pairs(NearGeom ng, const int* __restrict__ coff,
                                                         const typename Vec4<R>::T* __restrict__ xq,
                                                         const R* __restrict__ tab,
                                                         const typename Vec4<R>::T* __restrict__ offtab,
                                                         typename Vec4<R>::T* __restrict__ fsort,
                                                         double* __restrict__ out) {
  using V4 = typename Vec4<R>::T;
  using R2 = typename std::conditional<std::is_same<R, float>::value, float2, double2>::type;
  constexpr int kQ = 64;  // queue ring per warp
  constexpr int KC = near_cand<R>();
  constexpr int NW = kThreads / 32;
  __shared__ int QJ[NW][kQ];  // candidate slots of the queued pairs
  __shared__ R2 TAB[kRadialPieces * (kMaxDeg + 1)];
  __shared__ double part[NW][7];
  __shared__ int HPRE[kNearMaxHome + 1];  // prefix sums of the home cells' atom counts
  __shared__ int HT[kNearMaxHome];        // neighbourhood index of each home cell
  __shared__ int HD[kNearMaxHome];        // its (h0, h1, h2) as h0 << 20 | h1 << 10 | h2
  extern __shared__ __align__(16) unsigned char near_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int* qj_w = QJ[warp];

  const int blk = blockIdx.x;
  const int k2 = blk % ng.nb[2], k1 = (blk / ng.nb[2]) % ng.nb[1], k0b = blk / (ng.nb[2] * ng.nb[1]);
  const int hb0 = min(ng.B[0], ng.nc[0] - k0b * ng.B[0]);
  const int hb1 = min(ng.B[1], ng.nc[1] - k1 * ng.B[1]);
  const int hb2 = min(ng.B[2], ng.nc[2] - k2 * ng.B[2]);
  const int R0 = ng.R[0], R1 = ng.R[1], R2c = ng.R[2];
  const int RY = hb1 + 2 * R1, RZ = hb2 + 2 * R2c;
  const int nreg = (hb0 + R0) * RY * RZ;
  const int nh = hb0 * hb1 * hb2;
  const int nrow = 1 + R1 + R0 * (2 * R1 + 1);  // forward rows of a home cell

  V4* CB = reinterpret_cast<V4*>(near_smem);
  R* FJ = reinterpret_cast<R*>(CB + KC);  // x, y, z sums: FJ[e * KC + k]
  V4* OFF = reinterpret_cast<V4*>(FJ + 3 * KC);
  int* CS = reinterpret_cast<int*>(OFF + nreg);  // first sorted index of each cell
  int* PRE = CS + nreg;                          // nreg + 1 prefix sums of the atom counts
  int2* ROWS = reinterpret_cast<int2*>(PRE + nreg + 2);  // [home cell][row]: candidates [a, b)

  for (int t = threadIdx.x; t < nreg; t += blockDim.x) {
    const int r0 = t / (RY * RZ), r1 = (t / RZ) % RY - R1, r2 = t % RZ - R2c;
    const int u0 = k0b * ng.B[0] + r0, u1 = k1 * ng.B[1] + r1, u2 = k2 * ng.B[2] + r2;
    const int w0 = ((u0 % ng.nc[0]) + ng.nc[0]) % ng.nc[0];
    const int w1 = ((u1 % ng.nc[1]) + ng.nc[1]) % ng.nc[1];
    const int w2 = ((u2 % ng.nc[2]) + ng.nc[2]) % ng.nc[2];
    const int wc = (w0 * ng.nc[1] + w1) * ng.nc[2] + w2;
    const int cs = coff[wc];
    CS[t] = cs;
    PRE[t] = coff[wc + 1] - cs;  // the count, scanned below
    OFF[t] = offtab[((r0 * (ng.B[1] + 2 * R1)) + r1 + R1) * (ng.B[2] + 2 * R2c) + r2 + R2c];
  }
  const int nd = ng.ndeg;
  for (int e = threadIdx.x; e < kRadialPieces * (nd + 1); e += blockDim.x) {
    const int pc = e / (nd + 1), k = e - pc * (nd + 1);
    R2 v;
    v.x = tab[pc * (nd + 1) + k];
    v.y = tab[(kRadialPieces + pc) * (nd + 1) + k];
    TAB[e] = v;
  }
  for (int e = threadIdx.x; e < 3 * KC; e += blockDim.x) FJ[e] = R(0);
  __syncthreads();
  if (warp == 0) {
    int carry = 0;
    for (int base = 0; base < nreg; base += 32) {
      const int t = base + lane;
      const int v = t < nreg ? PRE[t] : 0;
      int x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      __syncwarp();
      if (t < nreg) PRE[t] = carry + x - v;
      carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) PRE[nreg] = carry;
    __syncwarp();
    // home cells in the order (h0, h1, h2): neighbourhood index and prefix sums of counts
    int v = 0, th = 0;
    if (lane < nh) {
      const int h0 = lane / (hb1 * hb2), h1 = (lane / hb2) % hb1, h2 = lane % hb2;
      th = (h0 * RY + h1 + R1) * RZ + h2 + R2c;
      v = PRE[th + 1] - PRE[th];
      HT[lane] = th;
      HD[lane] = h0 << 20 | h1 << 10 | h2;
    }
    int x = v;
#pragma unroll
    for (int o = 1; o < kNearMaxHome; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane < nh) HPRE[lane] = x - v;
    if (lane == nh - 1) HPRE[nh] = x;
  }
  __syncthreads();
  // forward rows of each home cell, numbered ro = 0 .. nrow - 1: row (0, 0) first (its
  // range starts after atom i), then (0, 1 .. R1), then (o0 >= 1, -R1 .. R1)
  for (int e = threadIdx.x; e < nh * nrow; e += blockDim.x) {
    const int h = e / nrow, ro = e - h * nrow;
    const int hd = HD[h];
    const int h0 = hd >> 20, h1 = (hd >> 10) & 1023, h2 = hd & 1023;
    int o0, o1;
    if (ro <= R1) {
      o0 = 0;
      o1 = ro;
    } else {
      o0 = 1 + (ro - R1 - 1) / (2 * R1 + 1);
      o1 = (ro - R1 - 1) % (2 * R1 + 1) - R1;
    }
    const int base = ((h0 + o0) * RY + h1 + o1 + R1) * RZ;
    ROWS[e] = make_int2(PRE[base + h2], PRE[base + h2 + 2 * R2c + 1]);
  }
  __syncthreads();
  const int total = PRE[nreg];
  const int nhome = HPRE[nh];
  if (nhome == 0) return;  // CTA-uniform
  const R rc2 = (R)(ng.rc * ng.rc), inv_rc = (R)ng.inv_rc;
  Sum<R> U, W[6];  // per lane over all of the warp's atoms

  for (int c0 = 0; c0 < total; c0 += KC) {
    const int kn = min(KC, total - c0);
    const int c1 = c0 + kn;
    if (c0 > 0) __syncthreads();  // the previous chunk's sums are flushed
    for (int t = warp; t < nreg; t += NW) {
      const int a = max(PRE[t], c0), b = min(PRE[t + 1], c1);
      if (a >= b) continue;
      const int jb = CS[t] + (a - PRE[t]);
      const V4 d = OFF[t];
      for (int k = a + lane; k < b; k += 32) {
        V4 xj = xq[jb + (k - a)];
        xj.x += d.x;
        xj.y += d.y;
        xj.z += d.z;
        CB[k - c0] = xj;
      }
    }
    __syncthreads();
    R u = R(0), w[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};  // plain sums over the chunk
    for (int hi = warp; hi < nhome; hi += NW) {
      const unsigned hm = __ballot_sync(0xffffffffu, lane < nh && HPRE[lane + 1] <= hi);
      const int h = __popc(hm);
      const int th = HT[h];
      const int rank = hi - HPRE[h];
      const int si = CS[th] + rank;  // sorted index of atom i
      const int ib = PRE[th] + rank;  // its slot in the neighbourhood
      const int2* rows = ROWS + h * nrow;
      V4 xi = xq[si];
      {
        const V4 d = OFF[th];
        xi.x += d.x;
        xi.y += d.y;
        xi.z += d.z;
      }
      R fx = R(0), fy = R(0), fz = R(0);
      // the warp alternates between filling its queue from the rows (until it holds 32
      // entries or the rows are done) and working 32 (or the last) entries
      int ro = 0;
      int ka = max(ib + 1, c0), kb = min(rows[0].y, c1);
      int qh = 0, qn = 0;  // queue head and length (warp-uniform)
      for (;;) {
        while (qn < 32) {
          if (ka >= kb) {
            if (++ro >= nrow) break;
            const int2 rr = rows[ro];
            ka = max(rr.x, c0);
            kb = min(rr.y, c1);
            continue;
          }
          const int k = ka + lane;
          bool pass = false;
          if (k < kb) {
            const V4 xj = CB[k - c0];
            const R dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
            const R r2 = dx * dx + dy * dy + dz * dz;
            pass = r2 > R(0) && r2 <= rc2;
          }
          const unsigned m = __ballot_sync(0xffffffffu, pass);
          if (pass) qj_w[(qh + qn + __popc(m & lt)) & (kQ - 1)] = k - c0;
          qn += __popc(m);
          ka += 32;
        }
        if (qn == 0) break;
        __syncwarp();
        const int mq = min(qn, 32);
        if (lane < mq) {
          const int js = qj_w[(qh + lane) & (kQ - 1)];
          const V4 e4 = CB[js];  // the same FP32 differences as the test above
          const R rx = xi.x - e4.x, ry = xi.y - e4.y, rz = xi.z - e4.z;
          const R r2 = rx * rx + ry * ry + rz * rz;
          R inv_r, r;
          if constexpr (std::is_same<R, float>::value) {
            inv_r = rsqrtf(r2);
            r = r2 * inv_r;
          } else {
            r = sqrt(r2);
            inv_r = R(1) / r;
          }
          R g1, g2;
          near_eval<ND>(TAB, nd, r * inv_rc, &g1, &g2);
          const R qq = xi.w * e4.w;
          const R en = qq * g1 * inv_r;
          const R f = qq * g2 * inv_r * inv_r * inv_r;
          const R px = f * rx, py = f * ry, pz = f * rz;
          fx += px;
          fy += py;
          fz += pz;
          atomicAdd(FJ + js, -px);
          atomicAdd(FJ + KC + js, -py);
          atomicAdd(FJ + 2 * KC + js, -pz);
          u += en;
          w[0] = fma(px, rx, w[0]);
          w[1] = fma(py, ry, w[1]);
          w[2] = fma(pz, rz, w[2]);
          w[3] = fma(px, ry, w[3]);
          w[4] = fma(px, rz, w[4]);
          w[5] = fma(py, rz, w[5]);
        }
        qh = (qh + mq) & (kQ - 1);
        qn -= mq;
        __syncwarp();  // the worked entries may be overwritten now
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
      }
      if (lane == 0) {
        if constexpr (std::is_same<R, float>::value) {
          red_add4(fsort + si, fx, fy, fz, 0.f);
        } else {
          R* fs = reinterpret_cast<R*>(fsort + si);
          atomicAdd(fs, fx);
          atomicAdd(fs + 1, fy);
          atomicAdd(fs + 2, fz);
        }
      }
    }
    U.add(u);
#pragma unroll
    for (int c = 0; c < 6; ++c) W[c].add(w[c]);
    __syncthreads();
    // the candidates' sums of this chunk go to the sorted-order accumulator
    for (int t = warp; t < nreg; t += NW) {
      const int a = max(PRE[t], c0), b = min(PRE[t + 1], c1);
      if (a >= b) continue;
      const int jb = CS[t] + (a - PRE[t]);
      for (int k = a + lane; k < b; k += 32) {
        const int s = k - c0;
        const R vx = FJ[s], vy = FJ[KC + s], vz = FJ[2 * KC + s];
        if (vx != R(0) || vy != R(0) || vz != R(0)) {
          FJ[s] = R(0);
          FJ[KC + s] = R(0);
          FJ[2 * KC + s] = R(0);
          if constexpr (std::is_same<R, float>::value) {
            red_add4(fsort + jb + (k - a), vx, vy, vz, 0.f);
          } else {
            R* fs = reinterpret_cast<R*>(fsort + jb + (k - a));
            atomicAdd(fs, vx);
            atomicAdd(fs + 1, vy);
            atomicAdd(fs + 2, vz);
          }
        }
      }
    }
  }
  double v[7] = {U.value(), W[0].value(), W[1].value(), W[2].value(),
                 W[3].value(), W[4].value(), W[5].value()};
#pragma unroll
  for (int e = 0; e < 7; ++e) {
    const double t = warp_sum(v[e]);
    if (lane == 0) part[warp][e] = t;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double t = 0.0;
    for (int w = 0; w < NW; ++w) t += part[w][threadIdx.x];
    if (t != 0.0) atomicAdd(out + threadIdx.x, t);
  }
}

// The step's results to page-locked host memory through its device mapping: nf floats
// (the first 4 * n16 as 16-byte words, coalesced) and nacc doubles of the accumulator.
__global__ void __launch_bounds__(kThreads) k_copy_out(const float* __restrict__ src,
                                                       float* __restrict__ dst, int64_t nf,
                                                       const double* __restrict__ acc,
                                                       double* __restrict__ acc_dst, int nacc) {
  const int64_t n16 = nf / 4;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int4* s4 = reinterpret_cast<const int4*>(src);
  int4* d4 = reinterpret_cast<int4*>(dst);
  for (int64_t i = tid; i < n16; i += nth) d4[i] = s4[i];
  for (int64_t i = 4 * n16 + tid; i < nf; i += nth) dst[i] = src[i];
  if (tid < nacc) acc_dst[tid] = acc[tid];
}

// Near forces from the sorted-order accumulator to the caller's array (input order):
// overwritten, or added to when add != 0.
template <typename R, typename IO>
__global__ void __launch_bounds__(kThreads) k_near_out(const int* __restrict__ coff, int ncells,
                                                       const int* __restrict__ idx,
                                                       const typename Vec4<R>::T* __restrict__ fsort,
                                                       IO* __restrict__ forces, int add) {
  const int ns = coff[ncells];
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
    const typename Vec4<R>::T f = fsort[s];
    IO* dst = forces + 3 * (int64_t)idx[s];
    if (add) {
      dst[0] = (IO)((double)dst[0] + (double)f.x);
      dst[1] = (IO)((double)dst[1] + (double)f.y);
      dst[2] = (IO)((double)dst[2] + (double)f.z);
    } else {
      dst[0] = (IO)f.x;
      dst[1] = (IO)f.y;
      dst[2] = (IO)f.z;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Fields on the grid from the kept spectrum X (Sec. 4.4 and Appendix C), one warp per
// spectrum row, lanes along i2, the same in-sphere decision as k_xfft:
//   KIND 0: G X                         (potential; per-atom energy)
//   KIND 1: i k_d G X, d = x, y, z      (eq. (rhodiagforce): ik-differentiation)
//   KIND 2: K_ab X / w^2, ab = xx yy zz xy xz yz, K = F I + (A x psi_0' / k^4 - 2 F / k^2) k k
//                                       (eq. (rhodiag): local pressure)
// G = F / w^2 with F = A psi_0(x) / k^2.  Modes outside the sphere are zero.  Field f of
// the output starts at out + f * M0 M1 H2.
template <typename R, int KIND>
__global__ void __launch_bounds__(kThreads) k_fields(const typename Cplx<R>::T* __restrict__ spec,
                                                     ScaleGeom s, const R* __restrict__ invw2,
                                                     const R* __restrict__ radtab,
                                                     typename Cplx<R>::T* __restrict__ out) {
  constexpr int NF = KIND == 0 ? 1 : (KIND == 1 ? 3 : 6);
  using C = typename Cplx<R>::T;
  const int lane = threadIdx.x & 31;
  const int nrows = s.M[0] * s.M[1];
  const int64_t Sz = (int64_t)nrows * s.H2;
  const ScaleConst<R> sc(s);
  const R* iw0 = invw2;
  const R* iw1 = invw2 + s.M[0];
  const R* iw2 = invw2 + s.M[0] + s.M[1];
  const int warps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int row = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); row < nrows; row += warps) {
    const int i0 = row / s.M[1];
    const int i1 = row - i0 * s.M[1];
    const int m0 = (2 * i0 <= s.M[0]) ? i0 : i0 - s.M[0];
    const int m1 = (2 * i1 <= s.M[1]) ? i1 : i1 - s.M[1];
    const bool rowin = abs(m0) <= s.mmax[0] && abs(m1) <= s.mmax[1];
    const R f0 = R(m0), f1 = R(m1);
    const R kx0 = f0 * bvec<R>(s, 0) + f1 * bvec<R>(s, 3);
    const R ky0 = f0 * bvec<R>(s, 1) + f1 * bvec<R>(s, 4);
    const R kz0 = f0 * bvec<R>(s, 2) + f1 * bvec<R>(s, 5);
    const R iw01 = iw0[i0] * iw1[i1];
    for (int i2 = lane; i2 < s.H2; i2 += 32) {
      const int m2 = i2;
      bool inside = rowin && m2 <= s.mmax[2] && (m0 | m1 | m2) != 0;
      R kx = R(0), ky = R(0), kz = R(0), k2 = R(0);
      if (inside) {
        const R f2 = R(m2);
        kx = kx0 + f2 * bvec<R>(s, 6);
        ky = ky0 + f2 * bvec<R>(s, 7);
        kz = kz0 + f2 * bvec<R>(s, 8);
        k2 = kx * kx + ky * ky + kz * kz;
        const R K2r = sc.K2;
        if (sizeof(R) == 8 || fabs(k2 - K2r) <= R(1e-5) * K2r) {
          const double dx = m0 * s.b[0] + m1 * s.b[3] + m2 * s.b[6];
          const double dy = m0 * s.b[1] + m1 * s.b[4] + m2 * s.b[7];
          const double dz = m0 * s.b[2] + m1 * s.b[5] + m2 * s.b[8];
          inside = dx * dx + dy * dy + dz * dz <= s.K2;
        } else {
          inside = k2 <= K2r;
        }
      }
      C o[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) o[f].x = o[f].y = R(0);
      if (inside) {
        const C X = spec[(int64_t)row * s.H2 + i2];
        const R iw = iw01 * iw2[i2];
        const R x = sqrt(k2) * sc.x_per_k;
        R psi, dpsi;
        radial_eval(radtab, s.rdeg, x, &psi, &dpsi);
        const R Fhat = sc.A * psi / k2;
        if constexpr (KIND == 0) {
          const R G = Fhat * iw;
          o[0].x = G * X.x;
          o[0].y = G * X.y;
        } else if constexpr (KIND == 1) {
          const R G = Fhat * iw;
          const R kk[3] = {kx, ky, kz};
#pragma unroll
          for (int d = 0; d < 3; ++d) {  // i t X = (-t X.y, t X.x)
            const R t = kk[d] * G;
            o[d].x = -t * X.y;
            o[d].y = t * X.x;
          }
        } else {
          const R dterm = sc.A * x * dpsi / (k2 * k2);
          const R cf = (dterm - R(2) * Fhat / k2) * iw;
          const R Fw = Fhat * iw;
          const R K[6] = {Fw + cf * kx * kx, Fw + cf * ky * ky, Fw + cf * kz * kz,
                          cf * kx * ky,      cf * kx * kz,      cf * ky * kz};
#pragma unroll
          for (int f = 0; f < 6; ++f) {
            o[f].x = K[f] * X.x;
            o[f].y = K[f] * X.y;
          }
        }
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) out[f * Sz + (int64_t)row * s.H2 + i2] = o[f];
    }
  }
}

// Window interpolation of NF (<= 3) real fields at the atoms: as k_gather (staged tile
// blocks, P lanes per atom, segmented shuffle), contracting with w0 w1 w2 only;
// out[idx * stride + off + f] = coef q_i sum_g field_f(g) w(g / M - s_i).
template <typename R, typename IO, int P, int NF>
__global__ void __launch_bounds__(kThreads, 2) k_gather_fields(
    Bins bins, TileGeom g, int ntiles, const R* __restrict__ wtab, const R* __restrict__ fields,
    int64_t field_stride, double coef, IO* __restrict__ out, int stride, int off) {
  using TC = TileC<P>;
  using V4 = typename Vec4<R>::T;
  const V4* __restrict__ sorted_tq = static_cast<const V4*>(bins.tq);
  const int* __restrict__ sorted_lb = bins.lb;
  const int* __restrict__ sorted_idx = bins.idx;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int E1 = TC::E1, E3p = TC::E3p, vol = TC::VOL, S1 = TC::S1;
  constexpr int PS = round_up4(P), RS = 3 * PS;
  R* phi = reinterpret_cast<R*>(smem_raw);  // NF blocks of vol
  const size_t wo = align32((size_t)NF * vol * sizeof(R));
  R* W = reinterpret_cast<R*>(smem_raw + wo);
  V4* TQ = reinterpret_cast<V4*>(smem_raw + wo + align32((size_t)kChunk * RS * sizeof(R)));
  int* B = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(TQ) + align32((size_t)kChunk * sizeof(V4)));
  int* X = B + kChunk;
  __shared__ int s_tile, s_cnt;
  const int E0 = g.E[0], E2 = g.E[2];
  constexpr int D = WinDeg<R>::value;
  constexpr int NP = kThreads / P;
  constexpr int G = 32 / P;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = lane / P, jj = lane - slot * P;
  const int p_t = threadIdx.x % P, pair0 = threadIdx.x / P;
  const bool evaluator = pair0 < NP;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const int t = atomicAdd(&bins.ctrl[5], 1);
      s_tile = t;
      if (t < ntiles) s_cnt = bins.tcount[t];
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile >= ntiles) break;
    const int start = tile * bins.cap, end = start + s_cnt;
    if (start == end) continue;
    const int t2 = tile % g.nt[2];
    const int t1 = (tile / g.nt[2]) % g.nt[1];
    const int t0 = tile / (g.nt[2] * g.nt[1]);
    const int o0 = t0 * g.T[0], o1 = t1 * g.T[1], o2 = t2 * g.T[2];
    {
      const int E1r = g.E[1];
      const int nload = E0 * E1r * E2;
      for (int e = threadIdx.x; e < NF * nload; e += blockDim.x) {
        const int f = e / nload, r = e - f * nload;
        const int c = r % E2;
        const int ab = r / E2;
        const int b = ab % E1r;
        const int a = ab / E1r;
        const int gi = wrap_index(o0 + a, g.M[0]);
        const int gj = wrap_index(o1 + b, g.M[1]);
        const int gk = wrap_index(o2 + c, g.M[2]);
        phi[f * vol + a * S1 + b * E3p + c] =
            fields[f * field_stride + ((int64_t)gi * g.M[1] + gj) * g.M[2] + gk];
      }
    }
    for (int c0 = start; c0 < end; c0 += kChunk) {
      const int cnt = min(kChunk, end - c0);
      for (int a = threadIdx.x; a < cnt; a += blockDim.x) {
        TQ[a] = sorted_tq[c0 + a];
        B[a] = local_base<S1, E3p>(sorted_lb[c0 + a]);
        X[a] = sorted_idx[c0 + a];
      }
      __syncthreads();
      if (evaluator) {
        R cw[D + 1];
#pragma unroll
        for (int k = 0; k <= D; ++k) cw[k] = __ldg(wtab + k * P + p_t);
        for (int pr = pair0; pr < 3 * cnt; pr += NP) {
          const int a = pr / 3, d = pr - 3 * a;
          W[a * RS + d * PS + p_t] = horner_reg<R, D>(cw, tq_comp<R>(TQ[a], d));
        }
      }
      __syncthreads();
      for (int a0 = warp * G; a0 < cnt; a0 += (kThreads / 32) * G) {
        const int a = a0 + slot;
        const bool valid = slot < G && a < cnt;
        R acc[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) acc[f] = R(0);
        if (valid) {
          const R* Wa = W + a * RS;
          R w0[P], w2[P];
          load_record<R, P>(Wa, w0);
          load_record<R, P>(Wa + 2 * PS, w2);
          const R w1 = Wa[PS + jj];
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const R* src = phi + f * vol + B[a] + jj * E3p;
            R sum = R(0);
#pragma unroll
            for (int kk = 0; kk < P; ++kk) {
              R sw = R(0);
#pragma unroll
              for (int i = 0; i < P; ++i) sw = fma(src[i * S1 + kk], w0[i], sw);
              sum = fma(w2[kk], sw, sum);
            }
            acc[f] = w1 * sum;
          }
        }
#pragma unroll
        for (int sft = 1; sft < P; sft <<= 1) {
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const R t = __shfl_down_sync(0xffffffffu, acc[f], sft);
            if (jj + sft < P) acc[f] += t;
          }
        }
        if (valid && jj == 0) {
          const double qa = (double)TQ[a].w;
#pragma unroll
          for (int f = 0; f < NF; ++f)
            out[(int64_t)X[a] * stride + off + f] = (IO)(coef * qa * (double)acc[f]);
        }
      }
      __syncthreads();
    }
  }

  // atoms past their tile's capacity: one warp per atom, straight from the global fields
  {
    const int novf = bins.ctrl[4];
    R* Ww = W + warp * (3 * kMaxP);
    const V4* otq = static_cast<const V4*>(bins.otq);
    for (;;) {
      int o = 0;
      if (lane == 0) o = atomicAdd(&bins.ctrl[6], 1);
      o = __shfl_sync(0xffffffffu, o, 0);
      if (o >= novf) break;
      const V4 v = otq[o];
      const int b0 = bins.ob[3 * o], b1 = bins.ob[3 * o + 1], b2 = bins.ob[3 * o + 2];
      for (int e = lane; e < 3 * P; e += 32) {
        const int d = e / P, pp = e - d * P;
        const R tau = tq_comp<R>(v, d) - R(0.5);
        R w = wtab[D * P + pp];
        for (int k = D - 1; k >= 0; --k) w = fma(w, tau, wtab[k * P + pp]);
        Ww[e] = w;
      }
      __syncwarp();
      R acc[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) acc[f] = R(0);
      for (int l = lane; l < P * P * P; l += 32) {
        const int i = l / (P * P), r = l - i * (P * P), j = r / P, k = r - j * P;
        const int gi = wrap_index(b0 + i, g.M[0]);
        const int gj = wrap_index(b1 + j, g.M[1]);
        const int gk = wrap_index(b2 + k, g.M[2]);
        const R w = Ww[i] * Ww[P + j] * Ww[2 * P + k];
#pragma unroll
        for (int f = 0; f < NF; ++f)
          acc[f] = fma(fields[f * field_stride + ((int64_t)gi * g.M[1] + gj) * g.M[2] + gk], w, acc[f]);
      }
#pragma unroll
      for (int sft = 16; sft > 0; sft >>= 1)
#pragma unroll
        for (int f = 0; f < NF; ++f) acc[f] += __shfl_xor_sync(0xffffffffu, acc[f], sft);
      if (lane == 0) {
        const int idx = bins.oidx[o];
#pragma unroll
        for (int f = 0; f < NF; ++f)
          out[(int64_t)idx * stride + off + f] = (IO)(coef * (double)v.w * (double)acc[f]);
      }
      __syncwarp();
    }
  }
  last_cta_resets(bins.ctrl, 7, 5, 3);
}

size_t fields_smem(bool fp64, int P, int NF) {
  int T[3], E3p, vol;
  tile_shape(P, T, &E3p, &vol);
  const size_t es = fp64 ? 8 : 4;
  const size_t rs = 3 * (size_t)round_up4(P);
  return align32((size_t)NF * vol * es) + align32(kChunk * rs * es) + align32(kChunk * 4 * es) +
         2 * kChunk * sizeof(int);
}

int grid_blocks(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (int)b;
}

// dispatch a functor templated on P
template <typename F>
cudaError_t with_P(int P, F&& f) {
  switch (P) {
    case 3: return f(std::integral_constant<int, 3>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 5: return f(std::integral_constant<int, 5>{});
    case 6: return f(std::integral_constant<int, 6>{});
    case 7: return f(std::integral_constant<int, 7>{});
    case 8: return f(std::integral_constant<int, 8>{});
    case 9: return f(std::integral_constant<int, 9>{});
    case 10: return f(std::integral_constant<int, 10>{});
    case 11: return f(std::integral_constant<int, 11>{});
    case 12: return f(std::integral_constant<int, 12>{});
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// ---- host launchers --------------------------------------------------------------------
// A launch with programmatic stream serialization (the kernel begins with pdl_wait), so
// its launch overlaps the end of the kernel before it; plain on the legacy default stream.
template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(void (*kern)(KArgs...), int grid, int block, size_t smem,
                       cudaStream_t st, Args... args) {
  if (st == nullptr) {
    kern<<<grid, block, smem, st>>>(args...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

cudaError_t launch_bin(bool io_double, bool fp64, const void* pos, const void* q, int64_t n,
                       const TileGeom& g, const Bins& b, void* bin_part_v, void* zero_buf,
                       size_t zero_bytes, cudaStream_t st) {
  if (n <= 0 || zero_bytes % 16 != 0) {
    if (zero_bytes) {
      const cudaError_t e = cudaMemsetAsync(zero_buf, 0, zero_bytes, st);
      if (e != cudaSuccess || n <= 0) return e;
    }
    zero_bytes = 0;
  }
  float2* bin_part = (float2*)bin_part_v;
  const int nb = grid_blocks(n);
  int4* zero = (int4*)zero_buf;
  const int64_t nzero = (int64_t)(zero_bytes / 16);
  if (io_double && fp64)
    k_bin<double, double><<<nb, kThreads, 0, st>>>((const double*)pos, (const double*)q, n, g, b,
                                                    bin_part, zero, nzero);
  else if (io_double)
    k_bin<double, float><<<nb, kThreads, 0, st>>>((const double*)pos, (const double*)q, n, g, b,
                                                   bin_part, zero, nzero);
  else if (fp64)
    k_bin<float, double><<<nb, kThreads, 0, st>>>((const float*)pos, (const float*)q, n, g, b,
                                                   bin_part, zero, nzero);
  else
    k_bin<float, float><<<nb, kThreads, 0, st>>>((const float*)pos, (const float*)q, n, g, b,
                                                  bin_part, zero, nzero);
  return cudaGetLastError();
}

int bin_blocks(int64_t n) { return grid_blocks(n); }

int bin_capacity(int64_t n, int ntiles) {
  const double mean = (double)std::max<int64_t>(n, 0) / std::max(ntiles, 1);
  int64_t cap = (int64_t)std::ceil(2.5 * mean) + 32;
  cap = (cap + 31) / 32 * 32;
  // slot indices stay within 32-bit ints; the overflow list takes the rest
  const int64_t most = ((int64_t)1 << 31) / std::max(ntiles, 1) / 32 * 32;
  return (int)std::max<int64_t>(32, std::min(cap, most));
}

size_t spread_smem_bytes(bool fp64, const TileGeom& g) {
  return spread_layout(fp64 ? 8 : 4, g.P).total;
}

size_t gather_smem_bytes(bool fp64, const TileGeom& g, bool bf16) {
  return gather_layout(fp64 ? 8 : 4, g.P, fp64 ? 8 : (bf16 ? 2 : 4)).total;
}

cudaError_t configure_kernels(bool fp64, int P, size_t spread_smem, size_t gather_smem,
                              bool bf16) {
  return with_P(P, [&](auto pc) -> cudaError_t {
    constexpr int PP = decltype(pc)::value;
    const int gs = (int)gather_smem;
    cudaError_t e;
    if (fp64) {
      e = cudaFuncSetAttribute(k_spread<double, PP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)spread_smem);
      if (e != cudaSuccess) return e;
      return cudaFuncSetAttribute(k_gather<double, double, PP, double>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, gs);
    }
    e = cudaFuncSetAttribute(k_spread<float, PP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)spread_smem);
    if (e != cudaSuccess) return e;
    if (bf16) {
      e = cudaFuncSetAttribute(k_gather<float, float, PP, __nv_bfloat16>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, gs);
      if (e != cudaSuccess) return e;
      return cudaFuncSetAttribute(k_gather<float, double, PP, __nv_bfloat16>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, gs);
    }
    e = cudaFuncSetAttribute(k_gather<float, float, PP, float>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, gs);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_gather<float, double, PP, float>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, gs);
  });
}

cudaError_t launch_spread(bool fp64, const TileGeom& g, int ntiles, int nblocks, const Bins& b,
                          const void* wtab, void* grid, cudaStream_t st) {
  const size_t smem = spread_smem_bytes(fp64, g);
  return with_P(g.P, [&](auto pc) -> cudaError_t {
    constexpr int PP = decltype(pc)::value;
    if (fp64)
      return pdl_launch(k_spread<double, PP>, nblocks, kThreads, smem, st, b, g, ntiles,
                        (const double*)wtab, (double*)grid);
    return pdl_launch(k_spread<float, PP>, nblocks, kThreads, smem, st, b, g, ntiles,
                      (const float*)wtab, (float*)grid);
  });
}

int xfft_blocks(const XGeom& x) { return (x.ncol + (1 << x.lognc) - 1) >> x.lognc; }

size_t xfft_smem_bytes(bool fp64, int M0, int lognc, int rdeg) {
  const size_t es = fp64 ? 8 : 4;
  return 2 * es * ((size_t)M0 + 2 * ((size_t)M0 << lognc)) +
         es * ((size_t)M0 + 2 * (size_t)kRadialPieces * (rdeg + 1));
}

namespace {
template <typename R>
cudaError_t set_xfft_smem(size_t smem) {
  cudaError_t e;
  const int b = (int)smem;
  if ((e = cudaFuncSetAttribute(k_xfft<R, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)))
    return e;
  if ((e = cudaFuncSetAttribute(k_xfft<R, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)))
    return e;
  if ((e = cudaFuncSetAttribute(k_xfft<R, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)))
    return e;
  return cudaFuncSetAttribute(k_xfft<R, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}
template <typename R>
cudaError_t run_xfft(bool fwd, bool inv, const XGeom& x, const ScaleGeom& s, const void* spec, void* out,
              const void* tw,
              const void* invw2, const void* radtab, double* partials, const int* order,
              const unsigned char* colact, int nactive, cudaStream_t st) {
  using C = typename Cplx<R>::T;
  const int nb = nactive;
  const size_t smem = xfft_smem_bytes(std::is_same<R, double>::value, x.M0, x.lognc, s.rdeg);
  // a plain launch: on the force path the kernel also waits for the side branch's clear
  auto go = [&](auto kern) {
    kern<<<nb, kXThreads, smem, st>>>((const C*)spec, (C*)out, x, s, (const C*)tw,
                                      (const R*)invw2, (const R*)radtab, partials, order, colact,
                                      nactive);
    return cudaGetLastError();
  };
  if (fwd && inv) return go(k_xfft<R, true, true>);
  if (fwd) return go(k_xfft<R, true, false>);
  if (inv) return go(k_xfft<R, false, true>);
  return go(k_xfft<R, false, false>);
}
}  // namespace

cudaError_t configure_xfft(bool fp64, size_t smem) {
  return fp64 ? set_xfft_smem<double>(smem) : set_xfft_smem<float>(smem);
}

cudaError_t launch_xfft(bool fp64, bool fwd, bool inv, const XGeom& x, const ScaleGeom& s,
                        const void* spec, void* out, const void* tw, const void* invw2,
                        const void* radtab,
                        double* partials, const int* order, const unsigned char* colact,
                        int nactive, cudaStream_t st) {
  if (nactive < 1) return cudaErrorInvalidValue;
  if (fp64)
    return run_xfft<double>(fwd, inv, x, s, spec, out, tw, invw2, radtab, partials, order, colact,
                            nactive, st);
  return run_xfft<float>(fwd, inv, x, s, spec, out, tw, invw2, radtab, partials, order, colact,
                         nactive, st);
}

size_t plane_smem_bytes(bool fp64, const PlaneGeom& pg) {
  return plane_smem_elems(pg) * (fp64 ? sizeof(double2) : sizeof(float2));
}

cudaError_t configure_planes(bool fp64, size_t smem) {
  const int b = (int)smem;
  cudaError_t e;
  if (fp64) {
    if ((e = cudaFuncSetAttribute(k_fplane<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)))
      return e;
    return cudaFuncSetAttribute(k_iplane<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  }
  if ((e = cudaFuncSetAttribute(k_fplane<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)))
    return e;
  if ((e = cudaFuncSetAttribute(k_iplane<float, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)))
    return e;
  return cudaFuncSetAttribute(k_iplane<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}

cudaError_t launch_fplane(bool fp64, const PlaneGeom& pg, const void* grid, void* box,
                          const void* tw, cudaStream_t st) {
  const size_t smem = plane_smem_bytes(fp64, pg);
  if (fp64)
    return pdl_launch(k_fplane<double>, pg.M0, plane_threads<double>(), smem, st, (const double*)grid,
                      (double2*)box, pg, (const double2*)tw);
  return pdl_launch(k_fplane<float>, pg.M0, plane_threads<float>(), smem, st, (const float*)grid,
                    (float2*)box, pg, (const float2*)tw);
}

cudaError_t launch_iplane(bool fp64, bool bf16, const PlaneGeom& pg, const void* box,
                          const unsigned char* colact, void* grid, const void* tw,
                          cudaStream_t st) {
  const size_t smem = plane_smem_bytes(fp64, pg);
  if (fp64)
    return pdl_launch(k_iplane<double, double>, pg.M0, plane_threads<double>(), smem, st,
                      (const double2*)box, colact, (double*)grid, pg, (const double2*)tw);
  if (bf16)
    return pdl_launch(k_iplane<float, __nv_bfloat16>, pg.M0, plane_threads<float>(), smem, st,
                      (const float2*)box, colact, (__nv_bfloat16*)grid, pg, (const float2*)tw);
  return pdl_launch(k_iplane<float, float>, pg.M0, plane_threads<float>(), smem, st,
                    (const float2*)box, colact, (float*)grid, pg, (const float2*)tw);
}

cudaError_t launch_copy_out(const void* src, void* dst, int64_t nf, const double* acc,
                            double* acc_dst, int nacc, int sms, cudaStream_t st) {
  k_copy_out<<<2 * sms, kThreads, 0, st>>>((const float*)src, (float*)dst, nf, acc, acc_dst, nacc);
  return cudaGetLastError();
}

cudaError_t launch_xsum(bool fp64, const double* partials, int nblk, const void* bin_part,
                        int nbin, double* accum, cudaStream_t st) {
  const float2* bp = (const float2*)bin_part;
  if (fp64)
    k_xsum<double><<<1, kThreads, 0, st>>>(partials, nblk, bp, nbin, accum);
  else
    k_xsum<float><<<1, kThreads, 0, st>>>(partials, nblk, bp, nbin, accum);
  return cudaGetLastError();
}

cudaError_t launch_gather(bool fp64, bool io_double, bool bf16, const GatherGeom& gg, int ntiles,
                          int nblocks, const Bins& b, const void* wtab, const void* grid,
                          void* forces, cudaStream_t st) {
  const size_t smem = gather_smem_bytes(fp64, gg.g, bf16);
  return with_P(gg.g.P, [&](auto pc) -> cudaError_t {
    constexpr int PP = decltype(pc)::value;
    if (fp64)
      return pdl_launch(k_gather<double, double, PP, double>, nblocks, kThreads, smem, st, b, gg,
                        ntiles, (const double*)wtab, (const double*)grid, (double*)forces);
    if (bf16) {
      const __nv_bfloat16* gb = (const __nv_bfloat16*)grid;
      if (io_double)
        return pdl_launch(k_gather<float, double, PP, __nv_bfloat16>, nblocks, kThreads, smem, st,
                          b, gg, ntiles, (const float*)wtab, gb, (double*)forces);
      return pdl_launch(k_gather<float, float, PP, __nv_bfloat16>, nblocks, kThreads, smem, st, b,
                        gg, ntiles, (const float*)wtab, gb, (float*)forces);
    }
    if (io_double)
      return pdl_launch(k_gather<float, double, PP, float>, nblocks, kThreads, smem, st, b, gg,
                        ntiles, (const float*)wtab, (const float*)grid, (double*)forces);
    return pdl_launch(k_gather<float, float, PP, float>, nblocks, kThreads, smem, st, b, gg, ntiles,
                      (const float*)wtab, (const float*)grid, (float*)forces);
  });
}

cudaError_t launch_cell_grad(bool io_double, const void* pos, const void* forces, int64_t n,
                             const CellGradArgs& c, const double* accum, double* grad,
                             cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(grad, 0, 9 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  const int nb = grid_blocks(n > 0 ? n : 1);
  if (io_double)
    k_cell_grad<double><<<nb, kThreads, 0, st>>>((const double*)pos, (const double*)forces, n, c,
                                                 accum, grad);
  else
    k_cell_grad<float><<<nb, kThreads, 0, st>>>((const float*)pos, (const float*)forces, n, c,
                                                accum, grad);
  return cudaGetLastError();
}

cudaError_t launch_near_bin(bool io_double, bool fp64, const void* pos, const void* q,
                            int64_t n, const NearGeom& ng, int* ccount, int* cell, int* rank,
                            void* xq_tmp, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int nb = grid_blocks(n);
  if (io_double && fp64)
    k_near_bin<double, double><<<nb, kThreads, 0, st>>>((const double*)pos, (const double*)q, n,
                                                        ng, ccount, cell, rank, (double4*)xq_tmp);
  else if (io_double)
    k_near_bin<double, float><<<nb, kThreads, 0, st>>>((const double*)pos, (const double*)q, n,
                                                       ng, ccount, cell, rank, (float4*)xq_tmp);
  else if (fp64)
    k_near_bin<float, double><<<nb, kThreads, 0, st>>>((const float*)pos, (const float*)q, n, ng,
                                                       ccount, cell, rank, (double4*)xq_tmp);
  else
    k_near_bin<float, float><<<nb, kThreads, 0, st>>>((const float*)pos, (const float*)q, n, ng,
                                                      ccount, cell, rank, (float4*)xq_tmp);
  return cudaGetLastError();
}

cudaError_t launch_near_scan(int* ccount, int* coff, int ncells, cudaStream_t st) {
  k_near_scan<<<1, kScanThreads, 0, st>>>(ccount, coff, ncells);
  return cudaGetLastError();
}

cudaError_t launch_near_scatter(bool fp64, int64_t n, const int* cell, const int* rank,
                                const int* coff, void* xq_tmp, void* xq, int* idx,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int nb = grid_blocks(n);
  if (fp64)
    k_near_scatter<double4><<<nb, kThreads, 0, st>>>(n, cell, rank, coff, (double4*)xq_tmp,
                                                     (double4*)xq, idx);
  else
    k_near_scatter<float4><<<nb, kThreads, 0, st>>>(n, cell, rank, coff, (float4*)xq_tmp,
                                                    (float4*)xq, idx);
  return cudaGetLastError();
}

int near_region_cells(const NearGeom& ng) {
  return (ng.B[0] + ng.R[0]) * (ng.B[1] + 2 * ng.R[1]) * (ng.B[2] + 2 * ng.R[2]);
}

size_t near_pairs_smem(bool fp64, const NearGeom& ng) {
  const int nrows = ng.B[0] * ng.B[1] * ng.B[2] * (1 + ng.R[1] + ng.R[0] * (2 * ng.R[1] + 1));
  return near_smem_bytes(fp64, near_region_cells(ng), nrows);
}

cudaError_t launch_near_pairs(bool fp64, bool io_double, const NearGeom& ng, int ncells,
                              const int* coff, const void* xq, const int* idx, const void* tab,
                              void* offtab, void* fsort, void* forces, int add, int64_t n,
                              double* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, 7 * sizeof(double), st);
  if (e != cudaSuccess || ncells <= 0 || n <= 0) return e;
  const int nreg = near_region_cells(ng);
  if (nreg > kNearMaxRegion) return cudaErrorInvalidValue;  // the host rejects such cells first
  const int nblocks = ng.nb[0] * ng.nb[1] * ng.nb[2];
  const size_t smem = near_pairs_smem(fp64, ng);
  if (smem > kNearMaxSmem) return cudaErrorInvalidValue;  // the host rejects such cells first
  if (fp64)
    k_near_offsets<double><<<(nreg + kThreads - 1) / kThreads, kThreads, 0, st>>>(ng, (double4*)offtab);
  else
    k_near_offsets<float><<<(nreg + kThreads - 1) / kThreads, kThreads, 0, st>>>(ng, (float4*)offtab);
  auto run = [&](auto kern, const auto* xqp, const auto* tabp, const auto* offp, auto* fsp) {
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (r != cudaSuccess) return r;
    kern<<<nblocks, kThreads, smem, st>>>(ng, coff, xqp, tabp, offp, fsp, out);
    return cudaGetLastError();
  };
  if (fp64) {
    e = run(k_near_pairs<double, 0>, (const double4*)xq, (const double*)tab, (const double4*)offtab,
            (double4*)fsort);
  } else {
    const float4* x4 = (const float4*)xq;
    const float* t = (const float*)tab;
    const float4* o4 = (const float4*)offtab;
    float4* f4 = (float4*)fsort;
    // the table degree as a compile-time constant where the FP32 fit usually lands
    switch (ng.ndeg) {
      case 6: e = run(k_near_pairs<float, 6>, x4, t, o4, f4); break;
      case 7: e = run(k_near_pairs<float, 7>, x4, t, o4, f4); break;
      case 8: e = run(k_near_pairs<float, 8>, x4, t, o4, f4); break;
      default: e = run(k_near_pairs<float, 0>, x4, t, o4, f4); break;
    }
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int nb = grid_blocks(n);
  if (fp64)
    k_near_out<double, double><<<nb, kThreads, 0, st>>>(coff, ncells, idx, (const double4*)fsort,
                                                        (double*)forces, add);
  else if (io_double)
    k_near_out<float, double><<<nb, kThreads, 0, st>>>(coff, ncells, idx, (const float4*)fsort,
                                                       (double*)forces, add);
  else
    k_near_out<float, float><<<nb, kThreads, 0, st>>>(coff, ncells, idx, (const float4*)fsort,
                                                      (float*)forces, add);
  return cudaGetLastError();
}

size_t fields_smem_bytes(bool fp64, int P, int NF) { return fields_smem(fp64, P, NF); }

cudaError_t launch_fields(bool fp64, int kind, const ScaleGeom& s, const void* spec,
                          const void* invw2, const void* radtab, void* out, cudaStream_t st) {
  const int rows = s.M[0] * s.M[1];
  const int nb = std::max(1, std::min((rows + kThreads / 32 - 1) / (kThreads / 32), 152 * 8));
  if (fp64) {
    using C = double2;
    if (kind == 0) k_fields<double, 0><<<nb, kThreads, 0, st>>>((const C*)spec, s, (const double*)invw2, (const double*)radtab, (C*)out);
    else if (kind == 1) k_fields<double, 1><<<nb, kThreads, 0, st>>>((const C*)spec, s, (const double*)invw2, (const double*)radtab, (C*)out);
    else k_fields<double, 2><<<nb, kThreads, 0, st>>>((const C*)spec, s, (const double*)invw2, (const double*)radtab, (C*)out);
  } else {
    using C = float2;
    if (kind == 0) k_fields<float, 0><<<nb, kThreads, 0, st>>>((const C*)spec, s, (const float*)invw2, (const float*)radtab, (C*)out);
    else if (kind == 1) k_fields<float, 1><<<nb, kThreads, 0, st>>>((const C*)spec, s, (const float*)invw2, (const float*)radtab, (C*)out);
    else k_fields<float, 2><<<nb, kThreads, 0, st>>>((const C*)spec, s, (const float*)invw2, (const float*)radtab, (C*)out);
  }
  return cudaGetLastError();
}

cudaError_t launch_gather_fields(bool fp64, bool io_double, const TileGeom& g, int ntiles,
                                 int nblocks, int nf, const Bins& b, const void* wtab,
                                 const void* fields, int64_t field_stride, double coef,
                                 void* out, int stride, int off, cudaStream_t st) {
  if (nf != 1 && nf != 3) return cudaErrorInvalidValue;
  const size_t smem = fields_smem(fp64, g.P, nf);
  return with_P(g.P, [&](auto pc) -> cudaError_t {
    constexpr int PP = decltype(pc)::value;
    auto go = [&](auto kernel, int /*unused*/, auto wt, auto fl, auto o) -> cudaError_t {
      cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      kernel<<<nblocks, kThreads, smem, st>>>(b, g, ntiles, wt, fl, field_stride, coef, o, stride, off);
      return cudaGetLastError();
    };
    if (fp64) {
      const int tq = 0;
      auto wt = (const double*)wtab;
      auto fl = (const double*)fields;
      return nf == 1 ? go(k_gather_fields<double, double, PP, 1>, tq, wt, fl, (double*)out)
                     : go(k_gather_fields<double, double, PP, 3>, tq, wt, fl, (double*)out);
    }
    const int tq = 0;
    auto wt = (const float*)wtab;
    auto fl = (const float*)fields;
    if (io_double)
      return nf == 1 ? go(k_gather_fields<float, double, PP, 1>, tq, wt, fl, (double*)out)
                     : go(k_gather_fields<float, double, PP, 3>, tq, wt, fl, (double*)out);
    return nf == 1 ? go(k_gather_fields<float, float, PP, 1>, tq, wt, fl, (float*)out)
                   : go(k_gather_fields<float, float, PP, 3>, tq, wt, fl, (float*)out);
  });
}

// resident CTAs per SM for the spread and gather kernels of this configuration
cudaError_t occupancy(bool fp64, bool io_double, int P, size_t spread_smem, size_t gather_smem,
                      int* spread_ctas, int* gather_ctas, bool bf16) {
  return with_P(P, [&](auto pc) -> cudaError_t {
    constexpr int PP = decltype(pc)::value;
    cudaError_t e;
    if (fp64) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(spread_ctas, k_spread<double, PP>, kThreads, spread_smem);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(gather_ctas, k_gather<double, double, PP, double>, kThreads, gather_smem);
      return e;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(spread_ctas, k_spread<float, PP>, kThreads, spread_smem);
    if (e != cudaSuccess) return e;
    if (bf16)
      return io_double ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(gather_ctas, k_gather<float, double, PP, __nv_bfloat16>, kThreads, gather_smem)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(gather_ctas, k_gather<float, float, PP, __nv_bfloat16>, kThreads, gather_smem);
    return io_double ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(gather_ctas, k_gather<float, double, PP, float>, kThreads, gather_smem)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(gather_ctas, k_gather<float, float, PP, float>, kThreads, gather_smem);
  });
}

}  // namespace esp
