/*
 * LSRN oracle, C part -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct CPU code that the tests, the smoke check and
 * the CPU-baseline leg of the benchmark use to judge the CUDA path.  Nothing in
 * the product library links, includes or calls this file, and this file
 * shares no code with the CUDA kernels.
 *
 * Contents
 *   1. Philox4x32-10 counter-based generator, restated from its published
 *      definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 *      easy as 1, 2, 3", SC'11, section on the Philox S-box): per round the
 *      two multipliers 0xD2511F53 / 0xCD9E8D57 act on words 0 and 2, the high
 *      halves are xor-ed with words 1 / 3 and the round key, and the key is
 *      bumped by the Weyl constants 0x9E3779B9 / 0xBB67AE85 between rounds.
 *   2. Box-Muller standard normals in binary32 with our own logarithm and
 *      sine/cosine (atanh series for log, Taylor series on [-pi/4, pi/4] for
 *      sin/cos; no libm transcendental is called), so that the normals are a
 *      fixed function of (seed, tag, i, j) that the GPU reproduces bit for
 *      bit.  Every step is one IEEE binary32 operation (round to nearest
 *      even); the file is compiled with -ffp-contract=off so that no
 *      multiply-add is fused behind our back, and fmaf is called where a
 *      fused operation is part of the definition.
 *   3. The sketching matrix G of Algorithms 1 and 2 (section 4.1): entry
 *      (i, j) is the normal above rounded to the grid 2^-12 (|G| < 8).
 *   4. One-sided (Hestenes) Jacobi SVD in FP64, cyclic-by-rows ordering,
 *      accumulating the right rotations -- the textbook algorithm (Golub and
 *      Van Loan, "Matrix Computations", one-sided Jacobi), used for the SVD
 *      steps of section 2.1 (x* = V Sigma^-1 U^T b) and of Algorithms 1/2
 *      step 4.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* 1. Philox4x32-10                                                          */
/* ------------------------------------------------------------------------ */

static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
  uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t y0 = hi1 ^ c[1] ^ k[0];
  uint32_t y2 = hi0 ^ c[3] ^ k[1];
  c[0] = y0;
  c[1] = lo1;
  c[2] = y2;
  c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int round = 0; round < 10; ++round) {
    philox_round(c, k);
    k[0] += 0x9E3779B9u;
    k[1] += 0xBB67AE85u;
  }
  out[0] = c[0];
  out[1] = c[1];
  out[2] = c[2];
  out[3] = c[3];
}

/* ------------------------------------------------------------------------ */
/* 2. binary32 uniforms, log, sin/cos(2 pi u), Box-Muller                    */
/* ------------------------------------------------------------------------ */

static float f32_from_bits(uint32_t b) {
  float f;
  memcpy(&f, &b, 4);
  return f;
}
static uint32_t bits_from_f32(float f) {
  uint32_t b;
  memcpy(&b, &f, 4);
  return b;
}

/* u = (2 * (x >> 9) + 1) * 2^-24: an odd multiple of 2^-24 in (0, 1), exact. */
float orc_uniform(uint32_t x) { return (float)(2u * (x >> 9) + 1u) * 0x1p-24f; }

/* Natural log for u in [2^-24, 1).  u = 2^e * f with f in [1/sqrt2, sqrt2);
 * ln f = 2 atanh(s), s = (f-1)/(f+1), |s| <= 0.1716, series to s^13. */
float orc_logf(float u) {
  uint32_t b = bits_from_f32(u);
  int e = (int)(b >> 23) - 127;
  float f = f32_from_bits((b & 0x007FFFFFu) | 0x3F800000u);
  if (f > f32_from_bits(0x3FB504F3u)) { /* sqrt(2) */
    f = f * 0.5f;
    e += 1;
  }
  float s = (f - 1.0f) / (f + 1.0f);
  float s2 = s * s;
  float p = fmaf(s2, f32_from_bits(0x3D9D89D9u), f32_from_bits(0x3DBA2E8Cu)); /* 1/13, 1/11 */
  p = fmaf(s2, p, f32_from_bits(0x3DE38E39u));                                /* 1/9 */
  p = fmaf(s2, p, f32_from_bits(0x3E124925u));                                /* 1/7 */
  p = fmaf(s2, p, f32_from_bits(0x3E4CCCCDu));                                /* 1/5 */
  p = fmaf(s2, p, f32_from_bits(0x3EAAAAABu));                                /* 1/3 */
  float t = s + s;
  float ts2 = t * s2;
  float lnf = fmaf(ts2, p, t);
  float ef = (float)e;
  float lo = fmaf(ef, f32_from_bits(0x35BFBE8Eu), lnf); /* ln2 low part */
  return fmaf(ef, f32_from_bits(0x3F317200u), lo);      /* ln2 high part */
}

/* sin and cos of 2 pi u for u in (0, 1): quarter-turn reduction that is exact
 * in binary32, then Taylor polynomials on |x| <= pi/4. */
void orc_sincos2pi(float u, float* sn, float* cs) {
  float t = u * 4.0f;
  int q = (int)t;
  float f = t - (float)q;
  if (f > 0.5f) {
    f = f - 1.0f;
    q += 1;
  }
  float x = f * f32_from_bits(0x3FC90FDBu); /* pi/2 */
  float x2 = x * x;
  float ps = fmaf(x2, f32_from_bits(0x3638EF1Du), f32_from_bits(0xB9500D01u)); /* 1/9!, -1/7! */
  ps = fmaf(x2, ps, f32_from_bits(0x3C088889u));                               /* 1/5! */
  ps = fmaf(x2, ps, f32_from_bits(0xBE2AAAABu));                               /* -1/3! */
  float x3 = x * x2;
  float sx = fmaf(x3, ps, x);
  float pc = fmaf(x2, f32_from_bits(0xB493F27Eu), f32_from_bits(0x37D00D01u)); /* -1/10!, 1/8! */
  pc = fmaf(x2, pc, f32_from_bits(0xBAB60B61u));                               /* -1/6! */
  pc = fmaf(x2, pc, f32_from_bits(0x3D2AAAABu));                               /* 1/4! */
  pc = fmaf(x2, pc, -0.5f);                                                    /* -1/2! */
  float cx = fmaf(x2, pc, 1.0f);
  switch (q & 3) {
    case 0: *sn = sx; *cs = cx; break;
    case 1: *sn = cx; *cs = -sx; break;
    case 2: *sn = -sx; *cs = -cx; break;
    default: *sn = -cx; *cs = sx; break;
  }
}

/* Standard normal for element (i, j) of the matrix drawn with (seed, tag).
 * One Philox call serves the four columns 4*floor(j/4) .. +3 of row i:
 * words (0,1) give the Box-Muller pair for columns +0 (cos) and +1 (sin),
 * words (2,3) the pair for columns +2 (cos) and +3 (sin). */
float orc_normal(uint64_t seed, uint32_t tag, uint64_t i, uint64_t j) {
  uint64_t q4 = j >> 2;
  uint32_t ctr[4] = {(uint32_t)q4, (uint32_t)(q4 >> 32), (uint32_t)i, tag};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  orc_philox4x32_10(ctr, key, w);
  int pair = (int)((j >> 1) & 1u);
  float u_r = orc_uniform(w[2 * pair]);
  float u_t = orc_uniform(w[2 * pair + 1]);
  float rad = sqrtf(-2.0f * orc_logf(u_r));
  float sn, cs;
  orc_sincos2pi(u_t, &sn, &cs);
  return (j & 1u) ? rad * sn : rad * cs;
}

/* G entry: the normal rounded to the grid 2^-12, clamped to |G| <= 32767/4096. */
static float quantize_g(float z) {
  float q = rintf(z * 4096.0f);
  if (q > 32767.0f) q = 32767.0f;
  if (q < -32767.0f) q = -32767.0f;
  return q * 0x1p-12f;
}

float orc_sketch_entry(uint64_t seed, uint32_t tag, uint64_t i, uint64_t j) {
  return quantize_g(orc_normal(seed, tag, i, j));
}

/* Fill a rows x cols row-major block of normals (z) and/or G entries (g),
 * covering matrix rows i0.. and columns j0..  Either output may be NULL. */
void orc_gauss_block(uint64_t seed, uint32_t tag, int64_t i0, int64_t j0, int64_t rows,
                     int64_t cols, float* z, double* g) {
  for (int64_t r = 0; r < rows; ++r) {
    for (int64_t c = 0; c < cols; ++c) {
      uint64_t i = (uint64_t)(i0 + r), j = (uint64_t)(j0 + c);
      float v = orc_normal(seed, tag, i, j);
      if (z) z[r * cols + c] = v;
      if (g) g[r * cols + c] = (double)quantize_g(v);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* 4. One-sided Jacobi SVD                                                   */
/* ------------------------------------------------------------------------ */

/* X is p x q, column-major with leading dimension ldx (column k at X + k*ldx).
 * V is q x q column-major (ldv), overwritten with the accumulated rotations
 * (starts from the identity).  On return the columns of X are mutually
 * orthogonal: X_out = X_in V, column k = sigma_k u_k.  sigma[k] = ||X_out[:,k]||.
 * No sorting is done here.  Returns the number of sweeps, or -1 if max_sweeps
 * were used without meeting |x_i . x_j| <= tol * ||x_i|| ||x_j|| for all pairs. */
int orc_jacobi_svd(int64_t p, int64_t q, double* X, int64_t ldx, double* V, int64_t ldv,
                   double* sigma, double tol, int max_sweeps) {
  for (int64_t j = 0; j < q; ++j)
    for (int64_t i = 0; i < q; ++i) V[j * ldv + i] = (i == j) ? 1.0 : 0.0;
  int sweeps = 0, converged = 0;
  while (!converged && sweeps < max_sweeps) {
    converged = 1;
    ++sweeps;
    for (int64_t a = 0; a < q - 1; ++a) {
      for (int64_t b = a + 1; b < q; ++b) {
        double* xa = X + a * ldx;
        double* xb = X + b * ldx;
        double aa = 0.0, bb = 0.0, ab = 0.0;
        for (int64_t k = 0; k < p; ++k) {
          aa += xa[k] * xa[k];
          bb += xb[k] * xb[k];
          ab += xa[k] * xb[k];
        }
        if (aa == 0.0 || bb == 0.0) continue;
        if (fabs(ab) <= tol * sqrt(aa) * sqrt(bb)) continue;
        converged = 0;
        double zeta = (bb - aa) / (2.0 * ab);
        double t;
        if (fabs(zeta) > 1e150) {
          t = 0.5 / zeta;
        } else {
          t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        }
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = c * t;
        for (int64_t k = 0; k < p; ++k) {
          double u = xa[k], w = xb[k];
          xa[k] = c * u - s * w;
          xb[k] = s * u + c * w;
        }
        double* va = V + a * ldv;
        double* vb = V + b * ldv;
        for (int64_t k = 0; k < q; ++k) {
          double u = va[k], w = vb[k];
          va[k] = c * u - s * w;
          vb[k] = s * u + c * w;
        }
      }
    }
  }
  for (int64_t j = 0; j < q; ++j) {
    double acc = 0.0;
    for (int64_t k = 0; k < p; ++k) acc += X[j * ldx + k] * X[j * ldx + k];
    sigma[j] = sqrt(acc);
  }
  return converged ? sweeps : -1;
}

/* ------------------------------------------------------------------------ */
/* 5. Residuals in double-double                                             */
/* ------------------------------------------------------------------------ */
/* Error-free transformations: two_sum (Knuth) and two_prod (via fma) give
 * s + e = a + b and p + e = a * b exactly; sums of such pairs carry about
 * 106 significant bits.  Used to compute least-squares residuals
 * r = b - A x and normal-equation residuals A^T r accurately enough that the
 * min-length solution of the stored A can be pinned below the FP64 floor. */
static void two_sum(double a, double b, double* s, double* e) {
  double t = a + b;
  double bb = t - a;
  *e = (a - (t - bb)) + (b - bb);
  *s = t;
}

static void dd_add_prod(double* hi, double* lo, double a, double b) {
  double p = a * b;
  double pe = fma(a, b, -p);
  double s, se;
  two_sum(*hi, p, &s, &se);
  double l = *lo + se + pe;
  double h2, l2;
  two_sum(s, l, &h2, &l2);
  *hi = h2;
  *lo = l2;
}

/* r = b - A x for row-major A (m x n, lda); result rounded to double. */
void orc_dd_residual(int64_t m, int64_t n, const double* A, int64_t lda, const double* b,
                     const double* x, double* r) {
  for (int64_t i = 0; i < m; ++i) {
    double hi = b[i], lo = 0.0;
    const double* a = A + i * lda;
    for (int64_t j = 0; j < n; ++j) dd_add_prod(&hi, &lo, -a[j], x[j]);
    r[i] = hi + lo;
  }
}

/* g = A^T r for row-major A (m x n, lda), accumulated in double-double. */
void orc_dd_atr(int64_t m, int64_t n, const double* A, int64_t lda, const double* r,
                double* g) {
  for (int64_t j = 0; j < n; ++j) {
    double hi = 0.0, lo = 0.0;
    for (int64_t i = 0; i < m; ++i) dd_add_prod(&hi, &lo, A[i * lda + j], r[i]);
    g[j] = hi + lo;
  }
}
