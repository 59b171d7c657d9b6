/*
 * mvp_oracle.c -- plain, slow CPU oracle for the Mixture-of-Volumetric-Primitives
 * ray march (Lombardi et al., "Mixture of Volumetric Primitives for Efficient Neural
 * Rendering", TOG 2021).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load this library. The product path (the CUDA library) never calls
 * it, shares no code, header or constant with it, and this file includes nothing
 * from the product.
 *
 * Floating point: every value (positions, interpolation, compositing, gradients) is
 * FP64. Three discrete decisions depend on floating point and are taken in the
 * kernel's FP32 precision with a fixed operation order (round-to-nearest; this file
 * is compiled with -ffp-contract=off, so a fused multiply-add happens only where
 * fmaf is written out):
 *   - the Morton code of a primitive centre (a quantised integer), and
 *   - the ray/box slab interval that decides which primitives a ray hits and which
 *     samples fall inside a primitive ("f32spec" membership), and
 *   - the voxel cell (floor of the voxel coordinate) a sample falls in, which
 *     decides where the trilinear derivative jumps.
 * The FP64 plain definition of membership (the sample's local coordinates lie in
 * [-1,1]^3) is available too; tests check that the two agree except on samples
 * within 1e-4 (local units) of a box face.
 *
 * Paper sections followed:
 *   Sec. 3.1.2  primitive = position t_k, rotation R_k, per-axis scale s_k, payload
 *               V_k in R^{4 x M^3} (RGB + opacity) on a uniform voxel grid.
 *   Sec. 3.2.1  trilinear payload sampling; per-ray list of intersected primitives;
 *               a sample only checks primitives of that list; data-parallel BVH
 *               (Karras) rebuilt every frame.
 *   Sec. 3.2.2  I_p = int V_col dT/dt dt, T(t) = min(int V_alpha dt, 1), A_p = T(t_max),
 *               early stop once T > 1 - eps_early, additive accumulation.
 *   Sec. 3.1.4  final composite with the background image (Eq. for I~ at the end of
 *               the "Background Model" paragraph).
 *
 * Readings where the paper is silent (each is stated where it is used):
 *   R1 quadrature: left Riemann sum on t_i = t_near + i*dt, i in [0, n_steps);
 *      per sample a = dt*sum_k alpha_k, c = dt*sum_k alpha_k*rgb_k,
 *      w = min(a, 1 - T), I += c*w/a, T += w  (T = min(sum a, 1) exactly).
 *   R2 several primitives at one sample: summed, then clamped once. The paper's
 *      literal rule, each primitive in turn in BVH order, is mode bit2
 *      (ORC_SEQUENTIAL): it differs only at a ray's saturating sample, where the
 *      primitives containing it are taken in the order of their Morton keys (the
 *      leaf order of the Karras hierarchy), each adding w_k = min(dt alpha_k, 1 - T)
 *      of its colour until T = 1.
 *   R3 s_k are half extents: x = t_k + R_k diag(s_k) y with y in [-1,1]^3.
 *   R4 corner-aligned voxels: u = (y+1)/2*(M-1), cell i0 = min(floor(u), M-2).
 *   R5 I_p is already weighted by dT, so the background composite is
 *      I~ = I + (1 - A) B. Mode bit3 (ORC_LITERAL) reads the printed composite
 *      literally instead: I~ = A I + (1 - A) B.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#pragma STDC FP_CONTRACT OFF

#define ORC_FACE_BAND 1e-4  /* |max_j |y_j| - 1| below this marks a near-face sample */
#define ORC_GRAZE_T 1e-4    /* |t_out - t_in| below this marks a grazing ray/box pair */

/* ------------------------------------------------------------------------- */
/* Sec. 3.1.2: R_k from the unit quaternion q/|q|, q = (w, x, y, z).           */
/* Row-major R[3*i + j]; a local point y maps to world t + R diag(s) y.        */
/* ------------------------------------------------------------------------- */
static void rot_f64(const float *q4, double R[9]) {
  double w = q4[0], x = q4[1], y = q4[2], z = q4[3];
  double n = sqrt(w * w + x * x + y * y + z * z);
  w /= n; x /= n; y /= n; z /= n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

void orc_rotations(int n, const float *q, double *R_out) {
  for (int k = 0; k < n; ++k) rot_f64(q + 4 * k, R_out + 9 * k);
}

/* The same rotation in FP32 with a fixed order of correctly rounded operations. */
static void rot_f32spec(const float *q4, float R[9]) {
  float q0 = q4[0], q1 = q4[1], q2 = q4[2], q3 = q4[3];
  float n2 = q0 * q0;
  n2 = n2 + q1 * q1;
  n2 = n2 + q2 * q2;
  n2 = n2 + q3 * q3;
  float nrm = sqrtf(n2);
  float w = q0 / nrm, x = q1 / nrm, y = q2 / nrm, z = q3 / nrm;
  float xx = x * x, yy = y * y, zz = z * z;
  float xy = x * y, xz = x * z, yz = y * z;
  float wx = w * x, wy = w * y, wz = w * z;
  R[0] = 1.0f - 2.0f * (yy + zz); R[1] = 2.0f * (xy - wz);        R[2] = 2.0f * (xz + wy);
  R[3] = 2.0f * (xy + wz);        R[4] = 1.0f - 2.0f * (xx + zz); R[5] = 2.0f * (yz - wx);
  R[6] = 2.0f * (xz - wy);        R[7] = 2.0f * (yz + wx);        R[8] = 1.0f - 2.0f * (xx + yy);
}

void orc_rotations_f32spec(int n, const float *q, float *R_out) {
  for (int k = 0; k < n; ++k) rot_f32spec(q + 4 * k, R_out + 9 * k);
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.2.1: which primitives a ray intersects, and over which t.            */
/* Slab method in the primitive's local frame, where the box is [-1,1]^3.      */
/* ------------------------------------------------------------------------- */

/* FP32 decision, fixed operation order, each step correctly rounded (fmaf is the
 * fused multiply-add with one rounding): p = o - t; per axis j
 * ol = fma(R2j, p2, fma(R1j, p1, R0j*p0)) * (1/s_j), dl likewise with d; a ray with
 * dl == 0 is inside the slab iff |ol| <= 1, else with r = 1/dl the slab spans
 * (-1 - ol)*r .. (1 - ol)*r. Returns 1 on a hit with [tin, tout]. */
static int slab_f32spec(const float R[9], const float *t, const float *s, const float *o,
                        const float *d, float t_near, float t_far, float *tin, float *tout) {
  float p0 = o[0] - t[0], p1 = o[1] - t[1], p2 = o[2] - t[2];
  float lo = t_near, hi = t_far;
  for (int j = 0; j < 3; ++j) {
    float is = 1.0f / s[j];
    float on = fmaf(R[2 * 3 + j], p2, fmaf(R[1 * 3 + j], p1, R[0 * 3 + j] * p0));
    float dn = fmaf(R[2 * 3 + j], d[2], fmaf(R[1 * 3 + j], d[1], R[0 * 3 + j] * d[0]));
    float ol = on * is;
    float dl = dn * is;
    if (dl == 0.0f) {
      if (ol < -1.0f || ol > 1.0f) return 0;
    } else {
      float r = 1.0f / dl;
      float t1 = (-1.0f - ol) * r;
      float t2 = (1.0f - ol) * r;
      lo = fmaxf(lo, fminf(t1, t2));
      hi = fminf(hi, fmaxf(t1, t2));
    }
  }
  *tin = lo;
  *tout = hi;
  return lo <= hi;
}

/* FP64 slab interval against the box |y_j| <= ext (ext = 1 is the primitive).
 * Returns tout - tin (negative: a miss by that much in t); -HUGE_VAL when a ray
 * parallel to a slab lies outside it. */
static double slab_f64(const double R[9], const float *t, const float *s, const float *o,
                       const float *d, double t_near, double t_far, double ext,
                       double *tin, double *tout) {
  double p[3] = {(double)o[0] - t[0], (double)o[1] - t[1], (double)o[2] - t[2]};
  double lo = t_near, hi = t_far;
  for (int j = 0; j < 3; ++j) {
    double ol = (R[0 * 3 + j] * p[0] + R[1 * 3 + j] * p[1] + R[2 * 3 + j] * p[2]) / s[j];
    double dl = (R[0 * 3 + j] * d[0] + R[1 * 3 + j] * d[1] + R[2 * 3 + j] * d[2]) / s[j];
    if (dl == 0.0) {
      if (fabs(ol) > ext) { *tin = lo; *tout = hi; return -HUGE_VAL; }
    } else {
      double t1 = (-ext - ol) / dl, t2 = (ext - ol) / dl;
      lo = fmax(lo, fmin(t1, t2));
      hi = fmin(hi, fmax(t1, t2));
    }
  }
  *tin = lo;
  *tout = hi;
  return hi - lo;
}

/* Per-ray hit counts. spec 0: FP64 pairs with tout - tin >= -ORC_GRAZE_T (hits plus
 * near misses, so callers can tell grazing pairs apart); spec 1: FP32 decision. */
void orc_hit_counts(int n, const float *t, const float *q, const float *s, int64_t n_rays,
                    const float *o, const float *d, float t_near, float t_far, int spec,
                    int64_t *counts) {
  double *R64 = (double *)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
  float *R32 = (float *)malloc(sizeof(float) * 9 * (size_t)(n > 0 ? n : 1));
  for (int k = 0; k < n; ++k) { rot_f64(q + 4 * k, R64 + 9 * k); rot_f32spec(q + 4 * k, R32 + 9 * k); }
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t r = 0; r < n_rays; ++r) {
    int64_t c = 0;
    for (int k = 0; k < n; ++k) {
      if (spec) {
        float a, b;
        c += slab_f32spec(R32 + 9 * k, t + 3 * k, s + 3 * k, o + 3 * r, d + 3 * r, t_near, t_far, &a, &b);
      } else {
        double a, b;
        c += slab_f64(R64 + 9 * k, t + 3 * k, s + 3 * k, o + 3 * r, d + 3 * r, t_near, t_far, 1.0, &a, &b) >= -ORC_GRAZE_T;
      }
    }
    counts[r] = c;
  }
  free(R64);
  free(R32);
}

/* Fill CSR hit lists (offs from the counts above), primitives in increasing k.
 * margin (nullable) receives tout - tin of each FP64 pair. */
void orc_hit_fill(int n, const float *t, const float *q, const float *s, int64_t n_rays,
                  const float *o, const float *d, float t_near, float t_far, int spec,
                  const int64_t *offs, int32_t *ids, double *tin, double *tout, double *margin) {
  double *R64 = (double *)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
  float *R32 = (float *)malloc(sizeof(float) * 9 * (size_t)(n > 0 ? n : 1));
  for (int k = 0; k < n; ++k) { rot_f64(q + 4 * k, R64 + 9 * k); rot_f32spec(q + 4 * k, R32 + 9 * k); }
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t r = 0; r < n_rays; ++r) {
    int64_t w = offs[r];
    for (int k = 0; k < n; ++k) {
      if (spec) {
        float a, b;
        if (slab_f32spec(R32 + 9 * k, t + 3 * k, s + 3 * k, o + 3 * r, d + 3 * r, t_near, t_far, &a, &b)) {
          ids[w] = k; tin[w] = a; tout[w] = b;
          if (margin) margin[w] = (double)b - (double)a;
          ++w;
        }
      } else {
        double a, b;
        double m = slab_f64(R64 + 9 * k, t + 3 * k, s + 3 * k, o + 3 * r, d + 3 * r, t_near, t_far, 1.0, &a, &b);
        if (m >= -ORC_GRAZE_T) {
          ids[w] = k; tin[w] = a; tout[w] = b;
          if (margin) margin[w] = m;
          ++w;
        }
      }
    }
  }
  free(R64);
  free(R32);
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.2.1 (Karras BVH): Morton keys of the primitive centres.              */
/* Scene bounds are the min/max of the centres; each axis is quantised to 10    */
/* bits in FP32 with a fixed order: u = (t - lo)/(hi - lo) (u = 0 if hi == lo), */
/* q = min(floor(u*1024), 1023); bits interleaved x,y,z from the top. The key   */
/* is (morton << 32) | k, which makes keys unique and the sort total.           */
/* ------------------------------------------------------------------------- */
static uint32_t spread10(uint32_t v) {
  uint32_t r = 0;
  for (int b = 0; b < 10; ++b) r |= ((v >> b) & 1u) << (3 * b);
  return r;
}

void orc_morton_keys(int n, const float *t, float *bounds6, uint64_t *keys) {
  float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int j = 0; j < 3; ++j) {
    if (n > 0) { lo[j] = t[j]; hi[j] = t[j]; }
    for (int k = 1; k < n; ++k) {
      lo[j] = fminf(lo[j], t[3 * k + j]);
      hi[j] = fmaxf(hi[j], t[3 * k + j]);
    }
    bounds6[j] = lo[j];
    bounds6[3 + j] = hi[j];
  }
  for (int k = 0; k < n; ++k) {
    uint32_t qv[3];
    for (int j = 0; j < 3; ++j) {
      float ext = hi[j] - lo[j];
      float u = ext > 0.0f ? (t[3 * k + j] - lo[j]) / ext : 0.0f;
      float f = floorf(u * 1024.0f);
      if (f > 1023.0f) f = 1023.0f;
      qv[j] = (uint32_t)f;
    }
    uint32_t m = (spread10(qv[0]) << 2) | (spread10(qv[1]) << 1) | spread10(qv[2]);
    keys[k] = ((uint64_t)m << 32) | (uint64_t)(uint32_t)k;
  }
}

/* Binary radix tree over sorted unique keys (the hierarchy of Karras 2012),
 * built top-down from its definition: the node covering [a, b] splits after the
 * last key whose bit at the first differing position of keys[a] and keys[b] is 0.
 * Node numbering of that construction: internal nodes 0..n-2 (root 0; a child
 * covering [a, g] is internal node g, one covering [g+1, b] is internal node g+1),
 * leaf j is node (n-1)+j. left/right hold the child node numbers. */
void orc_radix_tree(int n, const uint64_t *keys, int32_t *left, int32_t *right) {
  if (n < 2) return;
  int32_t *sa = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)n);
  int sp = 0;
  sa[0] = 0; sa[1] = n - 1; sa[2] = 0;  /* (a, b, node) */
  sp = 1;
  while (sp > 0) {
    --sp;
    int a = sa[3 * sp], b = sa[3 * sp + 1], node = sa[3 * sp + 2];
    uint64_t x = keys[a] ^ keys[b];
    int bit = 63;
    while (!((x >> bit) & 1ull)) --bit;  /* highest differing bit; keys are unique */
    int g = a;
    while (g + 1 <= b && !((keys[g + 1] >> bit) & 1ull)) ++g;
    int lc = (g == a) ? (n - 1) + g : g;
    int rc = (g + 1 == b) ? (n - 1) + g + 1 : g + 1;
    left[node] = lc;
    right[node] = rc;
    if (g != a) { sa[3 * sp] = a; sa[3 * sp + 1] = g; sa[3 * sp + 2] = g; ++sp; }
    if (g + 1 != b) { sa[3 * sp] = g + 1; sa[3 * sp + 1] = b; sa[3 * sp + 2] = g + 1; ++sp; }
  }
  free(sa);
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.2.1 / 3.2.2: the ray march.                                          */
/* ------------------------------------------------------------------------- */

typedef struct {
  int n, M;
  const float *t, *q, *s, *payload; /* payload FP32 [n][M][M][M][4], x fastest */
  double *R64;
  float *R32;
  float *U32; /* [n][3][4] FP32 voxel-coordinate rows, see voxel_coord_f32 */
  int *rank;  /* position of each primitive in the sorted Morton keys (mode bit2), or NULL */
} scene_t;

#define ORC_SEQUENTIAL 4
#define ORC_LITERAL 8 /* composite A I + (1 - A) B instead of I + (1 - A) B */

/* One primitive's trilinear RGBA at the current sample (sequential blending). */
typedef struct {
  int k;
  double v[4];
} seq_t;

typedef struct {
  const float *o, *d;
  float t_near, t_far, dt, eps;
  float bg[3];
  int n_steps;
} march_t;

/* FP32 sample time t_i = t_near + i*dt (product rounded, then the sum). */
static float sample_t_f32(const march_t *m, int i) {
  float p = (float)i * m->dt;
  return m->t_near + p;
}

/* The voxel cell of a sample is an integer decided by floating point; in the FP32
 * decision mode it is taken with the kernel's FP32 arithmetic: per primitive
 * hs_j = h/s_j (h = (M-1)/2), rows M_jm = hs_j R_mj and c_j = ((h - M_j0 t0) - M_j1 t1)
 * - M_j2 t2, each operation rounded; per sample x = fma(t_i, d, o) and
 * u_j = fma(M_j0, x0, fma(M_j1, x1, fma(M_j2, x2, c_j))). The cell is
 * min(floor(clamp(u, 0, M-1)), M-2) and an axis where u left [0, M-1] has zero
 * derivative. Values (weights, colours, gradients) stay FP64. */
static void voxel_rows_f32(const float R[9], const float *t, const float *s, int M, float rows[12]) {
  float h = 0.5f * (float)(M - 1);
  for (int j = 0; j < 3; ++j) {
    float hs = h / s[j];
    float c = h;
    for (int m = 0; m < 3; ++m) {
      float mj = hs * R[3 * m + j];
      rows[4 * j + m] = mj;
      float pr = mj * t[m];
      c = c - pr;
    }
    rows[4 * j + 3] = c;
  }
}

static void voxel_coord_f32(const float rows[12], const float *o, const float *d, float ti32, float u[3]) {
  float x0 = fmaf(ti32, d[0], o[0]), x1 = fmaf(ti32, d[1], o[1]), x2 = fmaf(ti32, d[2], o[2]);
  for (int j = 0; j < 3; ++j)
    u[j] = fmaf(rows[4 * j], x0, fmaf(rows[4 * j + 1], x1, fmaf(rows[4 * j + 2], x2, rows[4 * j + 3])));
}

/* Local coordinates y = diag(1/s) R^T (x - t) (R3). */
static void local_f64(const scene_t *sc, int k, const double x[3], double y[3]) {
  const double *R = sc->R64 + 9 * k;
  const float *t = sc->t + 3 * k, *s = sc->s + 3 * k;
  double p0 = x[0] - t[0], p1 = x[1] - t[1], p2 = x[2] - t[2];
  for (int j = 0; j < 3; ++j) y[j] = (R[0 * 3 + j] * p0 + R[1 * 3 + j] * p1 + R[2 * 3 + j] * p2) / s[j];
}

/* Trilinear RGBA at local coordinates y (R4), with the voxel coordinate clamped
 * to [0, M-1] (a no-op for samples inside the box). Optionally returns the 8 cell
 * corner voxel indices, their weights and dv/du (4 channels x 3 axes; zero along a
 * clamped axis). */
static void trilinear(const scene_t *sc, int k, const double y[3], const float *u32, double v[4],
                      int64_t cidx[8], double cw[8], double dvdu[4][3]) {
  int M = sc->M;
  double u[3], f[3];
  int i0[3], clamped[3];
  for (int j = 0; j < 3; ++j) {
    u[j] = (y[j] + 1.0) * 0.5 * (double)(M - 1);
    clamped[j] = 0;
    if (u[j] < 0.0) { u[j] = 0.0; clamped[j] = 1; }
    if (u[j] > (double)(M - 1)) { u[j] = (double)(M - 1); clamped[j] = 1; }
    if (u32) {  /* cell and clamp decided by the FP32 coordinate */
      float uf = u32[j];
      clamped[j] = !(uf >= 0.0f && uf <= (float)(M - 1));
      if (uf < 0.0f) uf = 0.0f;
      if (uf > (float)(M - 1)) uf = (float)(M - 1);
      int fl = (int)uf;
      i0[j] = fl < M - 2 ? fl : M - 2;
    } else {
      int fl = (int)floor(u[j]);
      i0[j] = fl < M - 2 ? fl : M - 2;
    }
    f[j] = u[j] - i0[j];
  }
  const float *P = sc->payload + (size_t)k * M * M * M * 4;
  for (int c = 0; c < 4; ++c) v[c] = 0.0;
  if (dvdu) for (int c = 0; c < 4; ++c) dvdu[c][0] = dvdu[c][1] = dvdu[c][2] = 0.0;
  for (int corner = 0; corner < 8; ++corner) {
    int bx = corner & 1, by = (corner >> 1) & 1, bz = (corner >> 2) & 1;
    double wx = bx ? f[0] : 1.0 - f[0];
    double wy = by ? f[1] : 1.0 - f[1];
    double wz = bz ? f[2] : 1.0 - f[2];
    double w = wx * wy * wz;
    int64_t vox = ((int64_t)(i0[2] + bz) * M + (i0[1] + by)) * M + (i0[0] + bx);
    const float *V = P + 4 * vox;
    for (int c = 0; c < 4; ++c) v[c] += w * (double)V[c];
    if (cidx) { cidx[corner] = vox; cw[corner] = w; }
    if (dvdu) {
      double sx = bx ? 1.0 : -1.0, sy = by ? 1.0 : -1.0, sz = bz ? 1.0 : -1.0;
      for (int c = 0; c < 4; ++c) {
        dvdu[c][0] += sx * wy * wz * (double)V[c];
        dvdu[c][1] += wx * sy * wz * (double)V[c];
        dvdu[c][2] += wx * wy * sz * (double)V[c];
      }
    }
  }
  if (dvdu)
    for (int j = 0; j < 3; ++j)
      if (clamped[j]) for (int c = 0; c < 4; ++c) dvdu[c][j] = 0.0;
}

/* Per-ray candidate list for the pruned mode: FP64 intervals of each box inflated
 * to |y| <= 1 + ORC_FACE_BAND (so near-face samples are still seen), and the FP32
 * decision interval. */
typedef struct {
  int k;
  double a, b;      /* inflated FP64 interval */
  int hit32;        /* FP32 decision */
  float tin, tout;  /* FP32 interval */
} cand_t;

static int ray_candidates(const scene_t *sc, const march_t *m, int64_t r, cand_t *out) {
  int nc = 0;
  for (int k = 0; k < sc->n; ++k) {
    double a, b;
    double mg = slab_f64(sc->R64 + 9 * k, sc->t + 3 * k, sc->s + 3 * k, m->o + 3 * r, m->d + 3 * r,
                         m->t_near, m->t_far, 1.0 + ORC_FACE_BAND, &a, &b);
    float ta = 0, tb = 0;
    int h = slab_f32spec(sc->R32 + 9 * k, sc->t + 3 * k, sc->s + 3 * k, m->o + 3 * r, m->d + 3 * r,
                         m->t_near, m->t_far, &ta, &tb);
    if (mg >= 0.0 || h) {
      out[nc].k = k; out[nc].a = a; out[nc].b = b;
      out[nc].hit32 = h; out[nc].tin = ta; out[nc].tout = tb;
      ++nc;
    }
  }
  return nc;
}

/* Per-ray result of the forward march, as needed by the adjoint. */
typedef struct {
  double rgb[3], T;
  int i_last;      /* last sample processed (the ray stops after it) */
  int i_clamp;     /* sample where w = 1 - T < a (saturation), or -1 */
  double rho[3];   /* c/a at i_clamp (sequential: the colour of the primitive whose weight was
                    * clamped there, or 0 if none was) */
  double beta;     /* (1 - T)/a at i_clamp (sequential: that primitive's weight) */
  int seq_k;       /* sequential: the primitive clamped at i_clamp, or -1 */
  int64_t n_eval;  /* (sample, primitive) evaluations */
  int near_face;
} ray_out_t;

/* Does primitive entry `c` contain the sample? f32 membership uses the FP32
 * interval and the FP32 sample time; f64 membership uses |y_j| <= 1. Sets the
 * near-face flag from the FP64 local coordinates either way. */
static int member(const scene_t *sc, const cand_t *c, int brute_k, int f32m, float ti32,
                  const double x[3], double y[3], int *near_face) {
  int k = c ? c->k : brute_k;
  local_f64(sc, k, x, y);
  double ym = fmax(fabs(y[0]), fmax(fabs(y[1]), fabs(y[2])));
  if (fabs(ym - 1.0) < ORC_FACE_BAND) *near_face = 1;
  if (f32m) {
    if (c) return c->hit32 && c->tin <= ti32 && ti32 <= c->tout;
    return 0; /* brute f32 handled by caller */
  }
  return ym <= 1.0;
}

/* March one ray (R1, R2). mode bit0: 1 = pruned (per-ray candidate list), 0 = brute
 * (every primitive at every sample). mode bit1: 1 = FP32 membership decision.
 * mode bit2: sequential BVH-order blending at the saturating sample (needs sc->rank
 * and a buffer seq of n entries). */
static void march_ray(const scene_t *sc, const march_t *m, int64_t r, int mode, cand_t *cands,
                      seq_t *seq, ray_out_t *res) {
  int pruned = mode & 1, f32m = (mode >> 1) & 1, sequential = (mode & ORC_SEQUENTIAL) && seq && sc->rank;
  int nc = 0;
  if (pruned || f32m) nc = ray_candidates(sc, m, r, cands);
  const float *o = m->o + 3 * r, *d = m->d + 3 * r;
  double T = 0.0, I[3] = {0, 0, 0};
  res->i_last = m->n_steps - 1;
  res->i_clamp = -1;
  res->rho[0] = res->rho[1] = res->rho[2] = 0.0;
  res->beta = 0.0;
  res->seq_k = -1;
  res->n_eval = 0;
  res->near_face = 0;
  int nk = pruned ? nc : sc->n;
  for (int i = 0; i < m->n_steps; ++i) {
    float ti32 = sample_t_f32(m, i);
    double ti = f32m ? (double)ti32 : (double)m->t_near + (double)i * (double)m->dt;
    double x[3] = {o[0] + ti * d[0], o[1] + ti * d[1], o[2] + ti * d[2]};
    double a = 0.0, c[3] = {0, 0, 0};
    int n_in = 0;
    for (int e = 0; e < nk; ++e) {
      double y[3];
      int in;
      if (pruned) {
        if (!(cands[e].hit32 && f32m) && !(ti >= cands[e].a && ti <= cands[e].b)) continue;
        in = member(sc, &cands[e], -1, f32m, ti32, x, y, &res->near_face);
      } else if (f32m) {
        /* brute force with FP32 membership: look the primitive up in the list */
        const cand_t *ce = NULL;
        for (int z = 0; z < nc; ++z) if (cands[z].k == e) { ce = &cands[z]; break; }
        if (ce) in = member(sc, ce, -1, 1, ti32, x, y, &res->near_face);
        else { in = 0; member(sc, NULL, e, 0, ti32, x, y, &res->near_face); }
      } else {
        in = member(sc, NULL, e, 0, ti32, x, y, &res->near_face);
      }
      if (!in) continue;
      int k = pruned ? cands[e].k : e;
      double v[4];
      float u32[3];
      if (f32m) voxel_coord_f32(sc->U32 + 12 * k, o, d, ti32, u32);
      trilinear(sc, k, y, f32m ? u32 : NULL, v, NULL, NULL, NULL);
      a += v[3];
      c[0] += v[3] * v[0]; c[1] += v[3] * v[1]; c[2] += v[3] * v[2];
      res->n_eval++;
      if (sequential) {
        seq[n_in].k = k;
        for (int ch = 0; ch < 4; ++ch) seq[n_in].v[ch] = v[ch];
        ++n_in;
      }
    }
    a *= m->dt;
    c[0] *= m->dt; c[1] *= m->dt; c[2] *= m->dt;
    double rem = 1.0 - T;
    if (a <= rem) {
      I[0] += c[0]; I[1] += c[1]; I[2] += c[2];
      T += a;
    } else if (sequential) {
      /* the saturating sample, primitive by primitive in BVH order (insertion sort
       * by rank, then w_k = min(dt alpha_k, 1 - T)) */
      for (int x1 = 1; x1 < n_in; ++x1) {
        seq_t cur = seq[x1];
        int y1 = x1 - 1;
        while (y1 >= 0 && sc->rank[seq[y1].k] > sc->rank[cur.k]) { seq[y1 + 1] = seq[y1]; --y1; }
        seq[y1 + 1] = cur;
      }
      res->rho[0] = res->rho[1] = res->rho[2] = 0.0;
      res->beta = 0.0;
      int last = -1; /* the last contributing primitive while none has been clamped */
      for (int e = 0; e < n_in && rem > 0.0; ++e) {
        double w = m->dt * seq[e].v[3];
        if (w >= rem) {  /* this primitive's weight is clamped to what is left */
          w = rem;
          res->seq_k = seq[e].k;
          res->rho[0] = seq[e].v[0]; res->rho[1] = seq[e].v[1]; res->rho[2] = seq[e].v[2];
          res->beta = w;
          last = -2;
        } else if (w > 0.0) {
          last = e;
        }
        I[0] += seq[e].v[0] * w; I[1] += seq[e].v[1] * w; I[2] += seq[e].v[2] * w;
        rem -= w;
      }
      if (last >= 0) { /* rounding left every weight below what was left: the last one */
        res->seq_k = seq[last].k;
        res->rho[0] = seq[last].v[0]; res->rho[1] = seq[last].v[1]; res->rho[2] = seq[last].v[2];
        res->beta = m->dt * seq[last].v[3];
      }
      res->i_clamp = i;
      T = 1.0;
    } else {
      double beta = rem / a;
      I[0] += c[0] * beta; I[1] += c[1] * beta; I[2] += c[2] * beta;
      res->i_clamp = i;
      res->rho[0] = c[0] / a; res->rho[1] = c[1] / a; res->rho[2] = c[2] / a;
      res->beta = beta;
      T = 1.0;
    }
    if (T >= 1.0 - (double)m->eps) { res->i_last = i; break; }
  }
  res->T = T;
  res->rgb[0] = I[0]; res->rgb[1] = I[1]; res->rgb[2] = I[2];
}

static int scene_init(scene_t *sc, int n, int M, const float *t, const float *q, const float *s,
                      const float *payload) {
  sc->n = n; sc->M = M; sc->t = t; sc->q = q; sc->s = s; sc->payload = payload;
  sc->rank = NULL;
  sc->R64 = (double *)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
  sc->R32 = (float *)malloc(sizeof(float) * 9 * (size_t)(n > 0 ? n : 1));
  sc->U32 = (float *)malloc(sizeof(float) * 12 * (size_t)(n > 0 ? n : 1));
  if (!sc->R64 || !sc->R32 || !sc->U32) return -1;
  for (int k = 0; k < n; ++k) {
    rot_f64(q + 4 * k, sc->R64 + 9 * k);
    rot_f32spec(q + 4 * k, sc->R32 + 9 * k);
    voxel_rows_f32(sc->R32 + 9 * k, t + 3 * k, s + 3 * k, M, sc->U32 + 12 * k);
  }
  return 0;
}

static void scene_free(scene_t *sc) { free(sc->R64); free(sc->R32); free(sc->U32); free(sc->rank); }

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* BVH order: rank[k] = position of primitive k's (unique) Morton key in ascending
 * order, i.e. its leaf position in the Karras hierarchy. */
static int scene_rank(scene_t *sc) {
  int n = sc->n;
  size_t nb = (size_t)(n > 0 ? n : 1);
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * nb);
  sc->rank = (int *)malloc(sizeof(int) * nb);
  if (!keys || !sc->rank) { free(keys); return -1; }
  float b6[6];
  orc_morton_keys(n, sc->t, b6, keys);
  qsort(keys, (size_t)n, sizeof(uint64_t), cmp_u64);
  for (int i = 0; i < n; ++i) sc->rank[(uint32_t)(keys[i] & 0xffffffffu)] = i;
  free(keys);
  return 0;
}

/* Render: out[r] = (I + (1 - A) bg, A) (R5); near_face, n_eval and the adjoint
 * state (i_last, i_clamp; beta: (1 - T)/a at i_clamp, or under the sequential rule the
 * clamped primitive's weight; clamp_k: that primitive, -1 if none) are optional.
 * Returns 0, or -1 on bad input. */
int orc_render(int n, int M, const float *t, const float *q, const float *s, const float *payload,
               int64_t n_rays, const float *o, const float *d, float t_near, float t_far, float dt,
               float eps, const float *bg, int n_steps, int mode, int n_threads, double *out,
               uint8_t *near_face, int64_t *n_eval, int32_t *i_last, int32_t *i_clamp, double *beta,
               int32_t *clamp_k) {
  if (n < 0 || M < 2 || n_rays < 0 || !(dt > 0) || n_steps < 0) return -1;
  scene_t sc;
  if (scene_init(&sc, n, M, t, q, s, payload)) return -1;
  march_t m = {o, d, t_near, t_far, dt, eps, {bg[0], bg[1], bg[2]}, n_steps};
  if ((mode & ORC_SEQUENTIAL) && scene_rank(&sc)) {
    scene_free(&sc);
    return -1;
  }
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
#pragma omp parallel
  {
    cand_t *cands = (cand_t *)malloc(sizeof(cand_t) * (size_t)(n > 0 ? n : 1));
    seq_t *seq = (seq_t *)malloc(sizeof(seq_t) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 16)
    for (int64_t r = 0; r < n_rays; ++r) {
      ray_out_t res;
      march_ray(&sc, &m, r, mode, cands, seq, &res);
      double A = res.T;
      for (int c = 0; c < 3; ++c)
        out[4 * r + c] = ((mode & ORC_LITERAL) ? A * res.rgb[c] : res.rgb[c]) + (1.0 - A) * (double)bg[c];
      out[4 * r + 3] = A;
      if (near_face) near_face[r] = (uint8_t)res.near_face;
      if (n_eval) n_eval[r] = res.n_eval;
      if (i_last) i_last[r] = res.i_last;
      if (i_clamp) i_clamp[r] = res.i_clamp;
      if (beta) beta[r] = res.beta;
      if (clamp_k) clamp_k[r] = res.seq_k;
    }
    free(cands);
    free(seq);
  }
  scene_free(&sc);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of the march (Sec. 3.2.2 says the additive form allows a backward    */
/* pass without storing the per-sample graph; the supplemental with its details */
/* is not available, so this is derived from R1/R2 directly).                   */
/*                                                                             */
/* With S the clamped sample (if any), rho = c_S/a_S, beta = (1 - T_S)/a_S:      */
/*   no clamp: dL/da_i = gA, dL/dc_i = gI for every processed sample;           */
/*   clamp at S: i < S: dL/da_i = -gI.rho, dL/dc_i = gI;                         */
/*               i = S: dL/da_S = -(gI.rho) beta, dL/dc_S = gI beta.             */
/* gI = dL/dI~, gA = dL/dA - gI.bg (background composite R5).                   */
/* Per primitive at a sample: a = dt sum alpha_k, c = dt sum alpha_k rgb_k, so   */
/*   dL/dalpha_k = dt (dL/da + dL/dc . rgb_k), dL/drgb_k = dt alpha_k dL/dc.      */
/* Those flow to the 8 cell voxels with the trilinear weights, and through       */
/* dv/du * (M-1)/2 to y = diag(1/s) R^T (x - t), then to t_k, s_k, R_k and q_k.  */
/* ------------------------------------------------------------------------- */
static void quat_grad_from_R(const float *q4, const double G[9], double gq[4]) {
  double w = q4[0], x = q4[1], y = q4[2], z = q4[3];
  double n = sqrt(w * w + x * x + y * y + z * z);
  w /= n; x /= n; y /= n; z /= n;
  /* derivatives of the nine entries of R(w,x,y,z) (row-major) */
  double gw = G[1] * (-2 * z) + G[2] * (2 * y) + G[3] * (2 * z) + G[5] * (-2 * x) + G[6] * (-2 * y) + G[7] * (2 * x);
  double gx = G[1] * (2 * y) + G[2] * (2 * z) + G[3] * (2 * y) + G[4] * (-4 * x) + G[5] * (-2 * w) +
              G[6] * (2 * z) + G[7] * (2 * w) + G[8] * (-4 * x);
  double gy = G[0] * (-4 * y) + G[1] * (2 * x) + G[2] * (2 * w) + G[3] * (2 * x) + G[5] * (2 * z) +
              G[6] * (-2 * w) + G[7] * (2 * z) + G[8] * (-4 * y);
  double gz = G[0] * (-4 * z) + G[1] * (-2 * w) + G[2] * (2 * x) + G[3] * (2 * w) + G[4] * (-4 * z) +
              G[5] * (2 * y) + G[6] * (2 * x) + G[7] * (2 * y);
  /* through the normalisation q_hat = q/|q| */
  double dot = w * gw + x * gx + y * gy + z * gz;
  gq[0] = (gw - w * dot) / n;
  gq[1] = (gx - x * dot) / n;
  gq[2] = (gy - y * dot) / n;
  gq[3] = (gz - z * dot) / n;
}

/* Gradients are accumulated (+=) into g_payload [n][M^3][4], g_t [n][3],
 * g_q [n][4], g_s [n][3], all FP64. grad_out [R][4] = dL/d(out). */
int orc_backward(int n, int M, const float *t, const float *q, const float *s, const float *payload,
                 int64_t n_rays, const float *o, const float *d, float t_near, float t_far, float dt,
                 float eps, const float *bg, int n_steps, int mode, int n_threads,
                 const double *grad_out, double *g_payload, double *g_t, double *g_q, double *g_s) {
  if (n < 0 || M < 2 || n_rays < 0 || !(dt > 0) || n_steps < 0) return -1;
  if (mode & ORC_LITERAL) return -1; /* premultiplied composite only */
  scene_t sc;
  if (scene_init(&sc, n, M, t, q, s, payload)) return -1;
  march_t m = {o, d, t_near, t_far, dt, eps, {bg[0], bg[1], bg[2]}, n_steps};
  const int sequential = (mode & ORC_SEQUENTIAL) != 0;
  if (sequential && scene_rank(&sc)) {
    scene_free(&sc);
    return -1;
  }
  double *gR = (double *)calloc(9 * (size_t)(n > 0 ? n : 1), sizeof(double));
  int pruned = mode & 1, f32m = (mode >> 1) & 1;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
#pragma omp parallel
  {
    cand_t *cands = (cand_t *)malloc(sizeof(cand_t) * (size_t)(n > 0 ? n : 1));
    seq_t *seqb = (seq_t *)malloc(sizeof(seq_t) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 16)
    for (int64_t r = 0; r < n_rays; ++r) {
      ray_out_t res;
      march_ray(&sc, &m, r, mode, cands, seqb, &res);
      int nc = (pruned || f32m) ? ray_candidates(&sc, &m, r, cands) : 0;
      const double *go = grad_out + 4 * r;
      double gI[3] = {go[0], go[1], go[2]};
      double gA = go[3] - (gI[0] * bg[0] + gI[1] * bg[1] + gI[2] * bg[2]);
      double gIrho = gI[0] * res.rho[0] + gI[1] * res.rho[1] + gI[2] * res.rho[2];
      const float *or_ = o + 3 * r, *dr = d + 3 * r;
      int nk = pruned ? nc : n;
      for (int i = 0; i <= res.i_last; ++i) {
        double ga, gc[3];
        if (res.i_clamp < 0) { ga = gA; gc[0] = gI[0]; gc[1] = gI[1]; gc[2] = gI[2]; }
        else if (i < res.i_clamp) { ga = -gIrho; gc[0] = gI[0]; gc[1] = gI[1]; gc[2] = gI[2]; }
        else if (i == res.i_clamp) {
          ga = -gIrho * res.beta;
          gc[0] = gI[0] * res.beta; gc[1] = gI[1] * res.beta; gc[2] = gI[2] * res.beta;
        } else break;
        float ti32 = sample_t_f32(&m, i);
        double ti = f32m ? (double)ti32 : (double)t_near + (double)i * (double)dt;
        double x[3] = {or_[0] + ti * dr[0], or_[1] + ti * dr[1], or_[2] + ti * dr[2]};
        for (int e = 0; e < nk; ++e) {
          double y[3];
          int dummy = 0, in;
          if (pruned) {
            if (!(cands[e].hit32 && f32m) && !(ti >= cands[e].a && ti <= cands[e].b)) continue;
            in = member(&sc, &cands[e], -1, f32m, ti32, x, y, &dummy);
          } else if (f32m) {
            const cand_t *ce = NULL;
            for (int z = 0; z < nc; ++z) if (cands[z].k == e) { ce = &cands[z]; break; }
            in = ce ? member(&sc, ce, -1, 1, ti32, x, y, &dummy) : 0;
          } else {
            in = member(&sc, NULL, e, 0, ti32, x, y, &dummy);
          }
          if (!in) continue;
          int k = pruned ? cands[e].k : e;
          double v[4], cw[8], dvdu[4][3];
          int64_t cidx[8];
          float u32[3];
          /* sequential rule at the saturating sample S, with J the primitive whose weight was
           * clamped (w_J = 1 - T - the weights before it): a primitive before J in BVH order
           * adds dt alpha c and takes dt alpha from w_J, so it is differentiated like a
           * sample before S (dL/da = -gI.c_J, dL/dc = gI); J adds w_J c_J and its alpha does
           * not change I (dL/dalpha = 0, dL/dc = w_J gI); primitives after J add nothing.
           * Samples before S see dL/da = -gI.c_J (through 1 - T); with no clamped primitive
           * c_J = 0. */
          int seq_role = 0; /* 0: summed rule; 1: before J; 2: J; 3: after J */
          if (sequential && res.i_clamp >= 0 && i == res.i_clamp) {
            if (res.seq_k < 0 || sc.rank[k] < sc.rank[res.seq_k]) seq_role = 1;
            else seq_role = k == res.seq_k ? 2 : 3;
          }
          if (seq_role == 3) continue;
          if (f32m) voxel_coord_f32(sc.U32 + 12 * k, or_, dr, ti32, u32);
          trilinear(&sc, k, y, f32m ? u32 : NULL, v, cidx, cw, dvdu);
          double ga_k = ga, gc_k[3] = {gc[0], gc[1], gc[2]};
          if (seq_role == 1) { ga_k = -gIrho; gc_k[0] = gI[0]; gc_k[1] = gI[1]; gc_k[2] = gI[2]; }
          double galpha = dt * (ga_k + gc_k[0] * v[0] + gc_k[1] * v[1] + gc_k[2] * v[2]);
          double gv[4] = {dt * v[3] * gc_k[0], dt * v[3] * gc_k[1], dt * v[3] * gc_k[2], galpha};
          if (seq_role == 2) {
            gv[0] = res.beta * gI[0]; gv[1] = res.beta * gI[1]; gv[2] = res.beta * gI[2]; gv[3] = 0.0;
          }
          double *GP = g_payload + (size_t)k * M * M * M * 4;
          for (int cn = 0; cn < 8; ++cn)
            for (int ch = 0; ch < 4; ++ch) {
#pragma omp atomic
              GP[4 * cidx[cn] + ch] += cw[cn] * gv[ch];
            }
          double gy[3];
          for (int j = 0; j < 3; ++j)
            gy[j] = (gv[0] * dvdu[0][j] + gv[1] * dvdu[1][j] + gv[2] * dvdu[2][j] + gv[3] * dvdu[3][j]) *
                    0.5 * (double)(M - 1);
          const double *R = sc.R64 + 9 * k;
          const float *tk = t + 3 * k, *sk = s + 3 * k;
          double p[3] = {x[0] - tk[0], x[1] - tk[1], x[2] - tk[2]};
          for (int i2 = 0; i2 < 3; ++i2) {
            double acc = 0.0;
            for (int j = 0; j < 3; ++j) acc += R[3 * i2 + j] * gy[j] / sk[j];
#pragma omp atomic
            g_t[3 * k + i2] -= acc;
          }
          for (int j = 0; j < 3; ++j) {
#pragma omp atomic
            g_s[3 * k + j] -= gy[j] * y[j] / sk[j];
          }
          for (int i2 = 0; i2 < 3; ++i2)
            for (int j = 0; j < 3; ++j) {
#pragma omp atomic
              gR[9 * k + 3 * i2 + j] += p[i2] * gy[j] / sk[j];
            }
        }
      }
    }
    free(cands);
    free(seqb);
  }
  for (int k = 0; k < n; ++k) {
    double gq4[4];
    quat_grad_from_R(q + 4 * k, gR + 9 * k, gq4);
    for (int c = 0; c < 4; ++c) g_q[4 * k + c] += gq4[c];
  }
  free(gR);
  scene_free(&sc);
  return 0;
}
