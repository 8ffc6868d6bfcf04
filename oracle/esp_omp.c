/*
 * Plain FP64 ESP long-range step with OpenMP (test and benchmark infrastructure: the CPU
 * baseline timed beside the GPU path on all host cores).  Only tests, the smoke check and
 * the benchmark's CPU legs may load it.  It shares no code with the CUDA library.
 *
 * The same four steps as the FP64 numpy oracle (oracle/esp_grid.py), written out in C:
 *   1. spreading (Sec. 4.1 Step 1): rho(g) = sum_j q_j prod_d w_d(g_d/M_d - s_jd), window
 *      w_d(u) = psi_0(u / omega_d), omega_d = P / (2 M_d) (Sec. 4.2), stencil of Sec. 4.3;
 *   2. a forward 3D FFT (a recursive mixed-radix 2/3/5 transform, plain DFT for other
 *      factors);
 *   3. diagonal scaling over |k| <= c / r_c, k != 0 (eqs. (diag), (PFfinal)):
 *      a = |X|^2 / (2 V Mtot^2 prod_d w^_d^2), U_F = sum a F^, W_F = sum a [F^ I +
 *      (A x psi_0'(x) / k^4 - 2 F^ / k^2) k k], F^ = A psi_0(x) / k^2, X <- (F^ / w^2) X;
 *   4. the inverse FFT and the gather with the window gradient (eq. (AD)):
 *      F_i = -h^{-T} dU/ds_i, dU/ds_i = -(q_i / (V Mtot^2)) sum_g phi(g) grad_u w.
 * psi_0 and psi_0' come as Legendre coefficients; w^_d(m) = int w_d(u) e^{-2 pi i m u} du
 * by 64-point Gauss-Legendre.  Parallel loops over atoms (spreading with atomic adds),
 * over FFT lines and over modes; nothing else is reorganised.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
  double re, im;
} cplx;

/* sum_k coef[k] P_k(x), Legendre recurrence */
static double legendre_sum(const double* coef, int n, double x) {
  double p0 = 1.0, p1 = x, s = coef[0];
  if (n > 1) s += coef[1] * p1;
  for (int k = 1; k + 1 < n; ++k) {
    const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    s += coef[k + 1] * p2;
    p0 = p1;
    p1 = p2;
  }
  return s;
}

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration */
static void gauss(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* ---- FFT: recursive mixed radix, out[k] = sum_j in[j * stride] e^{sign 2 pi i j k / n}.
 * tw[t] = e^{2 pi i t / N} for the top-level length N (n divides N); out and scratch hold
 * n values each and do not overlap. */
static cplx twiddle(const cplx* tw, int N, int n, int64_t x, int sign) {
  const cplx t = tw[(x % n) * (N / n)];
  cplx r = {t.re, sign * t.im};
  return r;
}

static void fft_rec(const cplx* in, int stride, int n, int sign, cplx* out, cplx* scratch,
                    const cplx* tw, int N) {
  if (n == 1) {
    out[0] = in[0];
    return;
  }
  int p = 0;
  if (n % 2 == 0) p = 2;
  else if (n % 3 == 0) p = 3;
  else if (n % 5 == 0) p = 5;
  if (p == 0) { /* plain DFT for any other length */
    for (int k = 0; k < n; ++k) {
      double re = 0.0, im = 0.0;
      for (int j = 0; j < n; ++j) {
        const cplx t = twiddle(tw, N, n, (int64_t)j * k, sign);
        const cplx a = in[(int64_t)j * stride];
        re += a.re * t.re - a.im * t.im;
        im += a.re * t.im + a.im * t.re;
      }
      out[k].re = re;
      out[k].im = im;
    }
    return;
  }
  const int m = n / p;
  /* transforms of the p decimated sequences (every p-th element) into scratch */
  for (int r = 0; r < p; ++r)
    fft_rec(in + (int64_t)r * stride, stride * p, m, sign, scratch + r * m, out, tw, N);
  for (int k = 0; k < m; ++k)
    for (int j = 0; j < p; ++j) {
      double re = 0.0, im = 0.0;
      for (int r = 0; r < p; ++r) {
        const cplx t = twiddle(tw, N, n, (int64_t)r * (k + j * m), sign);
        const cplx a = scratch[r * m + k];
        re += a.re * t.re - a.im * t.im;
        im += a.re * t.im + a.im * t.re;
      }
      out[k + j * m].re = re;
      out[k + j * m].im = im;
    }
}

/* in-place 3D transform of a [M0][M1][M2] array, one dimension at a time */
static void fft3(cplx* a, const int* M, int sign) {
  for (int d = 2; d >= 0; --d) {
    const int n = M[d];
    const int64_t stride = d == 2 ? 1 : (d == 1 ? M[2] : (int64_t)M[1] * M[2]);
    const int64_t lines = (int64_t)M[0] * M[1] * M[2] / n;
    cplx* tw = (cplx*)malloc(sizeof(cplx) * n);
    for (int t = 0; t < n; ++t) {
      tw[t].re = cos(2.0 * M_PI * t / n);
      tw[t].im = sin(2.0 * M_PI * t / n);
    }
#pragma omp parallel
    {
      cplx* line = (cplx*)malloc(sizeof(cplx) * n);
      cplx* out = (cplx*)malloc(sizeof(cplx) * n);
      cplx* scr = (cplx*)malloc(sizeof(cplx) * n);
#pragma omp for schedule(static)
      for (int64_t L = 0; L < lines; ++L) {
        /* first element of line L along dimension d */
        int64_t base;
        if (d == 2) base = L * n;
        else if (d == 1) base = (L / M[2]) * (int64_t)M[1] * M[2] + (L % M[2]);
        else base = L;
        for (int j = 0; j < n; ++j) line[j] = a[base + j * stride];
        fft_rec(line, 1, n, sign, out, scr, tw, n);
        for (int j = 0; j < n; ++j) a[base + j * stride] = out[j];
      }
      free(line);
      free(out);
      free(scr);
    }
    free(tw);
  }
}

/* stencil base and the P window values (and u-derivatives) of grid coordinate x */
static int stencil(double x, int P, const double* coef, const double* dcoef, int nc, double* w,
                   double* dw, double dscale) {
  const int base = (P % 2 == 0) ? (int)floor(x) - P / 2 + 1 : (int)floor(x + 0.5) - (P - 1) / 2;
  for (int p = 0; p < P; ++p) {
    const double u = ((double)(base + p) - x) / (0.5 * P);
    w[p] = legendre_sum(coef, nc, u);
    if (dw) dw[p] = legendre_sum(dcoef, nc, u) * dscale;
  }
  return base;
}

static int wrap(int i, int m) {
  i %= m;
  return i < 0 ? i + m : i;
}

int esp_omp_step(int64_t n, const double* pos, const double* q, const double* h, const int* M,
                 int P, double c, double rc, int nc, const double* coef, const double* dcoef,
                 double lam0, double C0, double* energy, double* virial, double* forces,
                 int nthreads) {
  if (n < 0 || P < 2 || P > 16 || nc < 1) return -1;
  if (nthreads > 0) omp_set_num_threads(nthreads);
  /* h row-major (columns = cell vectors): inverse and volume */
  const double V = h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
                   h[2] * (h[3] * h[7] - h[4] * h[6]);
  if (!(V > 0.0)) return -2;
  double hi[9];
  hi[0] = (h[4] * h[8] - h[5] * h[7]) / V;
  hi[1] = (h[2] * h[7] - h[1] * h[8]) / V;
  hi[2] = (h[1] * h[5] - h[2] * h[4]) / V;
  hi[3] = (h[5] * h[6] - h[3] * h[8]) / V;
  hi[4] = (h[0] * h[8] - h[2] * h[6]) / V;
  hi[5] = (h[2] * h[3] - h[0] * h[5]) / V;
  hi[6] = (h[3] * h[7] - h[4] * h[6]) / V;
  hi[7] = (h[1] * h[6] - h[0] * h[7]) / V;
  hi[8] = (h[0] * h[4] - h[1] * h[3]) / V;
  const int64_t Mtot = (int64_t)M[0] * M[1] * M[2];
  double* rho = (double*)calloc(Mtot, sizeof(double));
  cplx* X = (cplx*)malloc(sizeof(cplx) * Mtot);
  if (!rho || !X) {
    free(rho);
    free(X);
    return -3;
  }

  /* 1. spreading */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double w[3][16];
    int b[3];
    for (int d = 0; d < 3; ++d) {
      double s = hi[3 * d] * pos[3 * i] + hi[3 * d + 1] * pos[3 * i + 1] + hi[3 * d + 2] * pos[3 * i + 2];
      s -= floor(s);
      if (s >= 1.0) s = 0.0;
      b[d] = stencil(M[d] * s, P, coef, dcoef, nc, w[d], NULL, 0.0);
    }
    for (int a = 0; a < P; ++a)
      for (int bb = 0; bb < P; ++bb) {
        const double qab = q[i] * w[0][a] * w[1][bb];
        const int64_t row = ((int64_t)wrap(b[0] + a, M[0]) * M[1] + wrap(b[1] + bb, M[1])) * M[2];
        for (int cc = 0; cc < P; ++cc) {
#pragma omp atomic
          rho[row + wrap(b[2] + cc, M[2])] += qab * w[2][cc];
        }
      }
  }

  /* 2. forward transform */
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < Mtot; ++g) {
    X[g].re = rho[g];
    X[g].im = 0.0;
  }
  fft3(X, M, -1);

  /* window transforms w^_d(m) = omega int_{-1}^{1} psi_0(t) cos(2 pi m omega t) dt */
  double gx[64], gw[64];
  gauss(64, gx, gw);
  double* what[3];
  for (int d = 0; d < 3; ++d) {
    what[d] = (double*)malloc(sizeof(double) * M[d]);
    const double om = 0.5 * P / M[d];
    for (int i = 0; i < M[d]; ++i) {
      const int m = (2 * i <= M[d]) ? i : i - M[d];
      double s = 0.0;
      for (int k = 0; k < 64; ++k) s += gw[k] * legendre_sum(coef, nc, gx[k]) * cos(2.0 * M_PI * m * om * gx[k]);
      what[d][i] = om * s;
    }
  }

  /* 3. scaling and reduction over |k| <= c / r_c */
  const double A = 2.0 * M_PI * lam0 / C0, K2 = (c / rc) * (c / rc);
  double U = 0.0, W[6] = {0, 0, 0, 0, 0, 0};
#pragma omp parallel for schedule(static) reduction(+ : U) reduction(+ : W[:6])
  for (int64_t g = 0; g < Mtot; ++g) {
    const int i0 = (int)(g / ((int64_t)M[1] * M[2])), i1 = (int)((g / M[2]) % M[1]), i2 = (int)(g % M[2]);
    const int m[3] = {(2 * i0 <= M[0]) ? i0 : i0 - M[0], (2 * i1 <= M[1]) ? i1 : i1 - M[1],
                      (2 * i2 <= M[2]) ? i2 : i2 - M[2]};
    double k[3];
    for (int e = 0; e < 3; ++e) k[e] = 2.0 * M_PI * (hi[e] * m[0] + hi[3 + e] * m[1] + hi[6 + e] * m[2]);
    const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    if ((m[0] == 0 && m[1] == 0 && m[2] == 0) || k2 > K2) {
      X[g].re = X[g].im = 0.0;
      continue;
    }
    const double x = sqrt(k2) * rc / c;
    const double Fh = A * legendre_sum(coef, nc, x) / k2;
    const double dterm = A * x * legendre_sum(dcoef, nc, x) / (k2 * k2);
    const double wp = what[0][i0] * what[1][i1] * what[2][i2];
    const double a = (X[g].re * X[g].re + X[g].im * X[g].im) / (2.0 * V * (double)Mtot * (double)Mtot * wp * wp);
    const double ck = a * (dterm - 2.0 * Fh / k2);
    U += a * Fh;
    W[0] += a * Fh + ck * k[0] * k[0];
    W[1] += a * Fh + ck * k[1] * k[1];
    W[2] += a * Fh + ck * k[2] * k[2];
    W[3] += ck * k[0] * k[1];
    W[4] += ck * k[0] * k[2];
    W[5] += ck * k[1] * k[2];
    const double G = Fh / (wp * wp);
    X[g].re *= G;
    X[g].im *= G;
  }
  *energy = U;
  virial[0] = W[0];
  virial[4] = W[1];
  virial[8] = W[2];
  virial[1] = virial[3] = W[3];
  virial[2] = virial[6] = W[4];
  virial[5] = virial[7] = W[5];

  /* 4. inverse transform and gather */
  if (forces) {
    fft3(X, M, +1);
    const double fs = 1.0 / (V * (double)Mtot * (double)Mtot);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      double w[3][16], dw[3][16];
      int b[3];
      for (int d = 0; d < 3; ++d) {
        double s = hi[3 * d] * pos[3 * i] + hi[3 * d + 1] * pos[3 * i + 1] + hi[3 * d + 2] * pos[3 * i + 2];
        s -= floor(s);
        if (s >= 1.0) s = 0.0;
        b[d] = stencil(M[d] * s, P, coef, dcoef, nc, w[d], dw[d], 2.0 * M[d] / P);
      }
      double g3[3] = {0, 0, 0};
      for (int a = 0; a < P; ++a)
        for (int bb = 0; bb < P; ++bb) {
          const int64_t row = ((int64_t)wrap(b[0] + a, M[0]) * M[1] + wrap(b[1] + bb, M[1])) * M[2];
          for (int cc = 0; cc < P; ++cc) {
            const double ph = X[row + wrap(b[2] + cc, M[2])].re;
            g3[0] += ph * dw[0][a] * w[1][bb] * w[2][cc];
            g3[1] += ph * w[0][a] * dw[1][bb] * w[2][cc];
            g3[2] += ph * w[0][a] * w[1][bb] * dw[2][cc];
          }
        }
      /* dU/ds = -(q / (V Mtot^2)) g3;  F = -h^{-T} dU/ds */
      for (int e = 0; e < 3; ++e)
        forces[3 * i + e] = q[i] * fs * (hi[e] * g3[0] + hi[3 + e] * g3[1] + hi[6 + e] * g3[2]);
    }
  }
  for (int d = 0; d < 3; ++d) free(what[d]);
  free(rho);
  free(X);
  return 0;
}
