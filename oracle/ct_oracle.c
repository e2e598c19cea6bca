/*
 * FP64 CPU oracle for the structure-tensor orientation pipeline.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may build, load or call this file.  It shares
 * no code, header, table or helper with the CUDA library, and the library
 * never calls it.
 *
 * What it computes (Summary; Figure 1b,c; Architecture, "orientation"): the 3D
 * structure tensor of an image volume, its eigen-decomposition, the eigenvector
 * of the smallest eigenvalue as the fibre direction, and helical angle (HA),
 * intrusion angle (IA) and fractional anisotropy (FA) in a cylindrical
 * left-ventricle frame, under an optional mask; volumes may be processed in
 * padded chunks (Implementation).  The paper prints no formulas, so each step
 * below is the textbook definition, with the reading taken where a choice is
 * needed stated beside it.  Everything is double precision and written as
 * plain loops; the only liberty taken is separability: a 3D Gaussian is the
 * product of 1D Gaussians, so each 3D filter is applied as three 1D passes
 * (identical in exact arithmetic to the triple sum; the tests check the two
 * against each other on small volumes).
 *
 * Anisotropic voxels (spacing (sx, sy, sz); reading stated where the paper is
 * silent): sigma, rho, the LV centre and axis are in the units of the
 * spacing; scale s along axis a becomes s / s_a voxels, gradient component a
 * is divided by s_a (the gradient in physical units), and positions are
 * (x sx, y sy, z sz).  An optional centreline gives slice z its own LV centre
 * (cx, cy, z sz).  Unit spacing without a centreline is the isotropic case.
 *
 * Conventions
 *   volume  vol[z][y][x], x fastest, uint16; dims = (nx, ny, nz)
 *   boxes   lo = (x0, y0, z0), n = (nx, ny, nz) in global voxel indices
 *   planes  SoA: component c of box voxel i at out[c * nvox + i]
 *   tensor  components (xx, yy, zz, xy, xz, yz)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CTO_OK 0
#define CTO_ERR_ARG (-1)
#define CTO_ERR_OOM (-2)
#define CTO_ERR_BOX (-3)

/* Truncation radius for scale s: R = floor(truncate * s + 0.5). */
int cto_radius(double s, double truncate) { return (int)floor(truncate * s + 0.5); }

/*
 * Sampled, normalised Gaussian and its derivative (taps k = -R..R, stored at
 * k + R):  w_k = exp(-k^2 / (2 s^2)) / sum_j exp(-j^2 / (2 s^2)),
 *          c_k = (k / s^2) w_k.
 * The gradient is the correlation g(x) = sum_k c_k I(x + k), i.e. the
 * convolution of I with d_k = -c_k, the derivative of the sampled Gaussian.
 */
int cto_kernels(double s, double truncate, double* w, double* c) {
  if (!(s > 0.0) || !(truncate > 0.0) || !w || !c) return CTO_ERR_ARG;
  int R = cto_radius(s, truncate);
  double sum = 0.0;
  for (int k = -R; k <= R; ++k) {
    w[k + R] = exp(-(double)k * (double)k / (2.0 * s * s));
    sum += w[k + R];
  }
  for (int k = -R; k <= R; ++k) {
    w[k + R] /= sum;
    c[k + R] = ((double)k / (s * s)) * w[k + R];
  }
  return CTO_OK;
}

typedef struct {
  int64_t lo[3];
  int64_t n[3];
} box_t;

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }
static int64_t box_vox(const box_t* b) { return b->n[0] * b->n[1] * b->n[2]; }

/* b grown by r[a] along each axis a, then clipped to the volume [0, dims). */
static box_t grow_clip3(const box_t* b, const int r[3], const int64_t dims[3]) {
  box_t o = *b;
  for (int a = 0; a < 3; ++a) {
    int64_t lo = b->lo[a] - r[a], hi = b->lo[a] + b->n[a] - 1 + r[a];
    if (lo < 0) lo = 0;
    if (hi > dims[a] - 1) hi = dims[a] - 1;
    o.lo[a] = lo;
    o.n[a] = hi - lo + 1;
  }
  return o;
}

/* b grown by r along one axis only, clipped. */
static box_t grow_axis(const box_t* b, int axis, int r, const int64_t dims[3]) {
  box_t o = *b;
  int64_t lo = clampi(b->lo[axis] - r, 0, dims[axis] - 1);
  int64_t hi = clampi(b->lo[axis] + b->n[axis] - 1 + r, 0, dims[axis] - 1);
  o.lo[axis] = lo;
  o.n[axis] = hi - lo + 1;
  return o;
}

static int box_inside(const box_t* in, const box_t* out) {
  for (int a = 0; a < 3; ++a)
    if (out->lo[a] < in->lo[a] || out->lo[a] + out->n[a] > in->lo[a] + in->n[a]) return 0;
  return 1;
}

/*
 * One 1D pass along `axis` with "nearest" boundary handling at the GLOBAL
 * volume edges (a coordinate beyond the volume is clamped to the edge voxel).
 * Inside the volume a box reads its true neighbours, which must lie in the
 * input box: that is the padded-chunk rule (Implementation).
 *   out(p) = sum_k taps[k + R] * in(clamp(p + k e_axis))          (odd = 0)
 *   out(p) = sum_{k>=1} taps[k + R] * (in(p + k) - in(p - k))       (odd = 1)
 * The odd form is the same sum for antisymmetric taps (c_-k = -c_k, c_0 = 0)
 * with each +k/-k pair taken together, so a constant input gives exactly 0.
 */
static int pass1d(const double* in, const box_t* ib, double* out, const box_t* ob, int axis, const double* taps,
                  int R, int odd, const int64_t dims[3]) {
  box_t need = grow_axis(ob, axis, R, dims);
  if (!box_inside(ib, &need)) return CTO_ERR_BOX;
  const int64_t sx = 1, sy = ib->n[0], sz = ib->n[0] * ib->n[1];
  const int64_t st = axis == 0 ? sx : (axis == 1 ? sy : sz);
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < ob->n[2]; ++z) {
    for (int64_t y = 0; y < ob->n[1]; ++y) {
      for (int64_t x = 0; x < ob->n[0]; ++x) {
        int64_t g[3] = {ob->lo[0] + x, ob->lo[1] + y, ob->lo[2] + z};
        int64_t base = (g[0] - ib->lo[0]) * sx + (g[1] - ib->lo[1]) * sy + (g[2] - ib->lo[2]) * sz;
        int64_t pa = g[axis];
        int64_t rel = pa - ib->lo[axis];
        double acc = 0.0;
        if (!odd) {
          for (int k = -R; k <= R; ++k) {
            int64_t q = clampi(pa + k, 0, dims[axis] - 1) - ib->lo[axis];
            acc += taps[k + R] * in[base + (q - rel) * st];
          }
        } else {
          for (int k = 1; k <= R; ++k) {
            int64_t qp = clampi(pa + k, 0, dims[axis] - 1) - ib->lo[axis];
            int64_t qm = clampi(pa - k, 0, dims[axis] - 1) - ib->lo[axis];
            acc += taps[k + R] * (in[base + (qp - rel) * st] - in[base + (qm - rel) * st]);
          }
        }
        out[(z * ob->n[1] + y) * ob->n[0] + x] = acc;
      }
    }
  }
  return CTO_OK;
}

static int check_box(const int64_t dims[3], const int64_t lo[3], const int64_t n[3]) {
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 1 || n[a] < 1 || lo[a] < 0 || lo[a] + n[a] > dims[a]) return CTO_ERR_ARG;
  }
  return CTO_OK;
}

/*
 * Gradient at noise scale sigma (Figure 1b; Architecture, "orientation"):
 *   g_x = c_x * w_y * w_z * I,  g_y = w_x * c_y * w_z * I,  g_z = w_x * w_y * c_z * I
 * each a separable filter applied z, then y, then x, with the kernels of
 * sig[a] (voxel units) along axis a (anisotropic voxels give a different
 * scale per axis).  Output: 3 planes over box, in voxel units.
 */
int cto_gradient3(const uint16_t* vol, const int64_t dims[3], const int64_t lo[3], const int64_t n[3],
                  const double sig[3], double truncate, double* g) {
  if (!vol || !g || check_box(dims, lo, n) || !(sig[0] > 0.0) || !(sig[1] > 0.0) || !(sig[2] > 0.0))
    return CTO_ERR_ARG;
  int R[3];
  double *w[3] = {NULL, NULL, NULL}, *c[3] = {NULL, NULL, NULL};
  for (int a = 0; a < 3; ++a) {
    R[a] = cto_radius(sig[a], truncate);
    w[a] = malloc(sizeof(double) * (2 * R[a] + 1));
    c[a] = malloc(sizeof(double) * (2 * R[a] + 1));
  }
  box_t ob = {{lo[0], lo[1], lo[2]}, {n[0], n[1], n[2]}};
  box_t ib = grow_clip3(&ob, R, dims);
  box_t bz = ib; /* after the z pass: x, y still padded, z = output range */
  bz.lo[2] = ob.lo[2];
  bz.n[2] = ob.n[2];
  box_t by = bz; /* after the y pass: x padded */
  by.lo[1] = ob.lo[1];
  by.n[1] = ob.n[1];
  double* I = malloc(sizeof(double) * box_vox(&ib));
  double* t1 = malloc(sizeof(double) * box_vox(&bz));
  double* t2 = malloc(sizeof(double) * box_vox(&by));
  int rc = CTO_OK;
  if (!w[0] || !w[1] || !w[2] || !c[0] || !c[1] || !c[2] || !I || !t1 || !t2) {
    rc = CTO_ERR_OOM;
    goto done;
  }
  for (int a = 0; a < 3; ++a) cto_kernels(sig[a], truncate, w[a], c[a]);
  for (int64_t z = 0; z < ib.n[2]; ++z)
    for (int64_t y = 0; y < ib.n[1]; ++y)
      for (int64_t x = 0; x < ib.n[0]; ++x)
        I[(z * ib.n[1] + y) * ib.n[0] + x] =
            (double)vol[((ib.lo[2] + z) * dims[1] + (ib.lo[1] + y)) * dims[0] + (ib.lo[0] + x)];
  int64_t nv = box_vox(&ob);
  for (int comp = 0; comp < 3; ++comp) {
    /* derivative along axis `comp`, smoothing along the other two */
    const double* tz = comp == 2 ? c[2] : w[2];
    const double* ty = comp == 1 ? c[1] : w[1];
    const double* tx = comp == 0 ? c[0] : w[0];
    if ((rc = pass1d(I, &ib, t1, &bz, 2, tz, R[2], comp == 2, dims))) goto done;
    if ((rc = pass1d(t1, &bz, t2, &by, 1, ty, R[1], comp == 1, dims))) goto done;
    if ((rc = pass1d(t2, &by, g + comp * nv, &ob, 0, tx, R[0], comp == 0, dims))) goto done;
  }
done:
  for (int a = 0; a < 3; ++a) {
    free(w[a]);
    free(c[a]);
  }
  free(I);
  free(t1);
  free(t2);
  return rc;
}

int cto_gradient(const uint16_t* vol, const int64_t dims[3], const int64_t lo[3], const int64_t n[3], double sigma,
                 double truncate, double* g) {
  const double sig[3] = {sigma, sigma, sigma};
  return cto_gradient3(vol, dims, lo, n, sig, truncate, g);
}

/*
 * Structure tensor at integration scale rho (Figure 1b; Implementation):
 *   J = g g^T (6 unique products), S_ab = G_rho * J_ab,
 * the rho-smoothing again separable (z, y, x) with "nearest" handling of the
 * PRODUCT field at the global edges.  Output: 6 planes (xx,yy,zz,xy,xz,yz) over
 * the box (lo, n).  The gradient is evaluated only where it is needed: on the
 * box grown by R_rho and clipped to the volume.
 * Per-axis form: sig[a] and rho3[a] are the scales along axis a in voxel
 * units, and gscale[a] multiplies gradient component a before the products
 * (1 / spacing[a] gives the gradient in physical units).
 */
int cto_structure_tensor3(const uint16_t* vol, const int64_t dims[3], const int64_t lo[3], const int64_t n[3],
                          const double sig[3], const double rho3[3], const double gscale[3], double truncate,
                          double* S) {
  if (!vol || !S || check_box(dims, lo, n)) return CTO_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (!(sig[a] > 0.0) || !(rho3[a] > 0.0)) return CTO_ERR_ARG;
  int Rr[3];
  double *w[3] = {NULL, NULL, NULL}, *c[3] = {NULL, NULL, NULL};
  for (int a = 0; a < 3; ++a) {
    Rr[a] = cto_radius(rho3[a], truncate);
    w[a] = malloc(sizeof(double) * (2 * Rr[a] + 1));
    c[a] = malloc(sizeof(double) * (2 * Rr[a] + 1));
  }
  box_t ob = {{lo[0], lo[1], lo[2]}, {n[0], n[1], n[2]}};
  box_t gb = grow_clip3(&ob, Rr, dims);
  box_t bz = gb;
  bz.lo[2] = ob.lo[2];
  bz.n[2] = ob.n[2];
  box_t by = bz;
  by.lo[1] = ob.lo[1];
  by.n[1] = ob.n[1];
  int64_t ng = box_vox(&gb), nv = box_vox(&ob);
  double* g = malloc(sizeof(double) * 3 * ng);
  double* J = malloc(sizeof(double) * ng);
  double* t1 = malloc(sizeof(double) * box_vox(&bz));
  double* t2 = malloc(sizeof(double) * box_vox(&by));
  int rc = CTO_OK;
  if (!g || !J || !t1 || !t2 || !w[0] || !w[1] || !w[2] || !c[0] || !c[1] || !c[2]) {
    rc = CTO_ERR_OOM;
    goto done;
  }
  if ((rc = cto_gradient3(vol, dims, gb.lo, gb.n, sig, truncate, g))) goto done;
  for (int a = 0; a < 3; ++a) cto_kernels(rho3[a], truncate, w[a], c[a]);
  static const int ca[6] = {0, 1, 2, 0, 0, 1};
  static const int cb[6] = {0, 1, 2, 1, 2, 2};
  for (int comp = 0; comp < 6; ++comp) {
    const double* ga = g + ca[comp] * ng;
    const double* gbb = g + cb[comp] * ng;
    const double sa = gscale[ca[comp]], sb = gscale[cb[comp]];
    for (int64_t i = 0; i < ng; ++i) J[i] = (sa * ga[i]) * (sb * gbb[i]);
    if ((rc = pass1d(J, &gb, t1, &bz, 2, w[2], Rr[2], 0, dims))) goto done;
    if ((rc = pass1d(t1, &bz, t2, &by, 1, w[1], Rr[1], 0, dims))) goto done;
    if ((rc = pass1d(t2, &by, S + comp * nv, &ob, 0, w[0], Rr[0], 0, dims))) goto done;
  }
done:
  free(g);
  free(J);
  free(t1);
  free(t2);
  for (int a = 0; a < 3; ++a) {
    free(w[a]);
    free(c[a]);
  }
  return rc;
}

int cto_structure_tensor(const uint16_t* vol, const int64_t dims[3], const int64_t lo[3], const int64_t n[3],
                         double sigma, double rho, double truncate, double* S) {
  const double sig[3] = {sigma, sigma, sigma}, rho3[3] = {rho, rho, rho}, one[3] = {1.0, 1.0, 1.0};
  return cto_structure_tensor3(vol, dims, lo, n, sig, rho3, one, truncate, S);
}

/*
 * Symmetric 3x3 eigen-decomposition by the cyclic Jacobi method (Golub & Van
 * Loan, Matrix Computations, section 8.5): sweep the pairs (0,1), (0,2), (1,2),
 * annihilating each off-diagonal entry with a plane rotation chosen by the
 * symmetric 2x2 Schur decomposition, until the off-diagonal Frobenius norm is
 * below 1e-15 of the whole norm.  Eigenvalues ascending in ev[0..2]; the unit
 * eigenvector of ev[k] in V[3k .. 3k+2].
 */
int cto_eig3(const double s6[6], double ev[3], double V[9]) {
  double A[3][3] = {{s6[0], s6[3], s6[4]}, {s6[3], s6[1], s6[5]}, {s6[4], s6[5], s6[2]}};
  double Q[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double fro = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) fro += A[i][j] * A[i][j];
  fro = sqrt(fro);
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = sqrt(2.0 * (A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2]));
    if (off <= 1e-15 * fro || off == 0.0) break;
    for (int p = 0; p < 2; ++p) {
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        double tau = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
        /* A <- J^T A J with J the rotation in the (p, q) plane */
        for (int k = 0; k < 3; ++k) {
          double akp = A[k][p], akq = A[k][q];
          A[k][p] = cs * akp - sn * akq;
          A[k][q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < 3; ++k) {
          double apk = A[p][k], aqk = A[q][k];
          A[p][k] = cs * apk - sn * aqk;
          A[q][k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          double qkp = Q[k][p], qkq = Q[k][q];
          Q[k][p] = cs * qkp - sn * qkq;
          Q[k][q] = sn * qkp + cs * qkq;
        }
      }
    }
  }
  int idx[3] = {0, 1, 2};
  double d[3] = {A[0][0], A[1][1], A[2][2]};
  for (int i = 0; i < 3; ++i) /* insertion sort, ascending */
    for (int j = i + 1; j < 3; ++j)
      if (d[idx[j]] < d[idx[i]]) {
        int t = idx[i];
        idx[i] = idx[j];
        idx[j] = t;
      }
  for (int k = 0; k < 3; ++k) {
    ev[k] = d[idx[k]];
    for (int r = 0; r < 3; ++r) V[3 * k + r] = Q[r][idx[k]];
  }
  return CTO_OK;
}

/* Eigenvalues (3 planes) and smallest-eigenvalue eigenvector (3 planes) of n tensors (6 planes). */
int cto_eig_field(const double* S, int64_t n, double* evals, double* v1) {
  if (!S || n < 0) return CTO_ERR_ARG;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s6[6], ev[3], V[9];
    for (int c = 0; c < 6; ++c) s6[c] = S[c * n + i];
    cto_eig3(s6, ev, V);
    for (int c = 0; c < 3; ++c) {
      if (evals) evals[c * n + i] = ev[c];
      if (v1) v1[c * n + i] = V[c];
    }
  }
  return CTO_OK;
}

/*
 * Fractional anisotropy of eigenvalues l1..l3 (Figure 1c), each clamped to
 * >= 0 (the tensor is positive semi-definite in exact arithmetic):
 *   FA = sqrt(1/2) * sqrt((l1-l2)^2 + (l2-l3)^2 + (l3-l1)^2) / sqrt(l1^2 + l2^2 + l3^2),
 * and FA = 0 where the denominator vanishes.
 */
double cto_fa(const double ev[3]) {
  double l1 = ev[0] > 0.0 ? ev[0] : 0.0, l2 = ev[1] > 0.0 ? ev[1] : 0.0, l3 = ev[2] > 0.0 ? ev[2] : 0.0;
  double den = l1 * l1 + l2 * l2 + l3 * l3;
  if (den == 0.0) return 0.0;
  double num = (l1 - l2) * (l1 - l2) + (l2 - l3) * (l2 - l3) + (l3 - l1) * (l3 - l1);
  return sqrt(0.5 * num / den);
}

/*
 * Helical and intrusion angle of fibre direction v at position p (Figure 1c):
 * the cylindrical frame about the left-ventricle centre c and axis a is
 *   e_z = a / |a|,  d = p - c,  r = d - (d . e_z) e_z,  e_r = r / |r|,  e_t = e_z x e_r.
 * With (v_r, v_t, v_z) the components of v in that frame, v is oriented so
 * that v_t > 0 (v_z >= 0 when v_t = 0), and
 *   HA = atan2(v_z, v_t)            (degrees, in (-90, 90])
 *   IA = asin(clamp(v_r, -1, 1))    (degrees: elevation out of the wall's tangent plane).
 * On the axis (|r| = 0) the frame does not exist: returns 0 and leaves HA, IA
 * to the caller's fill value.  `vo` receives the oriented v.
 */
int cto_ha_ia(const double p[3], const double c[3], const double a[3], const double v[3], double* ha, double* ia,
              double vo[3]) {
  double an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  double ez[3] = {a[0] / an, a[1] / an, a[2] / an};
  double d[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
  double h = d[0] * ez[0] + d[1] * ez[1] + d[2] * ez[2];
  double r[3] = {d[0] - h * ez[0], d[1] - h * ez[1], d[2] - h * ez[2]};
  double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  if (rn == 0.0) return 0;
  double er[3] = {r[0] / rn, r[1] / rn, r[2] / rn};
  double et[3] = {ez[1] * er[2] - ez[2] * er[1], ez[2] * er[0] - ez[0] * er[2], ez[0] * er[1] - ez[1] * er[0]};
  double vr = v[0] * er[0] + v[1] * er[1] + v[2] * er[2];
  double vt = v[0] * et[0] + v[1] * et[1] + v[2] * et[2];
  double vz = v[0] * ez[0] + v[1] * ez[1] + v[2] * ez[2];
  double sgn = (vt < 0.0 || (vt == 0.0 && vz < 0.0)) ? -1.0 : 1.0;
  vr *= sgn;
  vt *= sgn;
  vz *= sgn;
  for (int k = 0; k < 3; ++k) vo[k] = sgn * v[k];
  double rad2deg = 180.0 / 3.14159265358979323846;
  *ha = atan2(vz, vt) * rad2deg;
  double s = vr > 1.0 ? 1.0 : (vr < -1.0 ? -1.0 : vr);
  *ia = asin(s) * rad2deg;
  return 1;
}

/*
 * Per-voxel outputs over a box: oriented fibre vector (3 planes), HA, IA, FA.
 * Voxels where mask (global-volume shaped, may be NULL) is 0 get `fill` in
 * every output; on the axis HA and IA get `fill`.  Where no frame exists the
 * vector is oriented with its largest-magnitude component positive.
 */
int cto_angles_field3(const double* v1, const double* evals, const int64_t dims[3], const int64_t lo[3],
                      const int64_t n[3], const double center[3], const double axis[3], const double spacing[3],
                      const double* centres, const uint8_t* mask, double fill, double* vout, double* ha, double* ia,
                      double* fa) {
  if (!v1 || !evals || check_box(dims, lo, n)) return CTO_ERR_ARG;
  if (axis[0] == 0.0 && axis[1] == 0.0 && axis[2] == 0.0) return CTO_ERR_ARG;
  int64_t nv = n[0] * n[1] * n[2];
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < n[2]; ++z) {
    for (int64_t y = 0; y < n[1]; ++y) {
      for (int64_t x = 0; x < n[0]; ++x) {
        int64_t i = (z * n[1] + y) * n[0] + x;
        int64_t gx = lo[0] + x, gy = lo[1] + y, gz = lo[2] + z;
        double v[3] = {v1[i], v1[nv + i], v1[2 * nv + i]};
        double ev[3] = {evals[i], evals[nv + i], evals[2 * nv + i]};
        /* physical position; the LV centre of this slice when a centreline is given */
        double p[3] = {(double)gx * spacing[0], (double)gy * spacing[1], (double)gz * spacing[2]};
        double cs[3] = {center[0], center[1], center[2]};
        if (centres) {
          cs[0] = centres[2 * gz];
          cs[1] = centres[2 * gz + 1];
          cs[2] = p[2];
        }
        double h = fill, a = fill, vo[3];
        if (!cto_ha_ia(p, cs, axis, v, &h, &a, vo)) {
          int m = 0;
          for (int k = 1; k < 3; ++k)
            if (fabs(v[k]) > fabs(v[m])) m = k;
          double s = v[m] < 0.0 ? -1.0 : 1.0;
          for (int k = 0; k < 3; ++k) vo[k] = s * v[k];
          h = fill;
          a = fill;
        }
        double f = cto_fa(ev);
        if (mask && !mask[(gz * dims[1] + gy) * dims[0] + gx]) {
          h = a = f = fill;
          vo[0] = vo[1] = vo[2] = fill;
        }
        if (vout) {
          vout[i] = vo[0];
          vout[nv + i] = vo[1];
          vout[2 * nv + i] = vo[2];
        }
        if (ha) ha[i] = h;
        if (ia) ia[i] = a;
        if (fa) fa[i] = f;
      }
    }
  }
  return CTO_OK;
}

int cto_angles_field(const double* v1, const double* evals, const int64_t dims[3], const int64_t lo[3],
                     const int64_t n[3], const double center[3], const double axis[3], const uint8_t* mask,
                     double fill, double* vout, double* ha, double* ia, double* fa) {
  const double one[3] = {1.0, 1.0, 1.0};
  return cto_angles_field3(v1, evals, dims, lo, n, center, axis, one, NULL, mask, fill, vout, ha, ia, fa);
}

/*
 * The whole per-voxel pipeline over the box (lo, n) of a volume: structure
 * tensor (6 planes), eigenvalues (3), oriented fibre vector (3), HA, IA, FA.
 * Any output pointer may be NULL except S.
 */
int cto_pipeline3(const uint16_t* vol, const int64_t dims[3], const int64_t lo[3], const int64_t n[3], double sigma,
                  double rho, double truncate, const double spacing[3], const double center[3], const double axis[3],
                  const double* centres, const uint8_t* mask, double fill, double* S, double* evals, double* vout,
                  double* ha, double* ia, double* fa) {
  double sig[3], rho3[3], gs[3];
  for (int a = 0; a < 3; ++a) {
    if (!(spacing[a] > 0.0)) return CTO_ERR_ARG;
    sig[a] = sigma / spacing[a];
    rho3[a] = rho / spacing[a];
    gs[a] = 1.0 / spacing[a];
  }
  int rc = cto_structure_tensor3(vol, dims, lo, n, sig, rho3, gs, truncate, S);
  if (rc) return rc;
  int64_t nv = n[0] * n[1] * n[2];
  double* ev = evals ? evals : malloc(sizeof(double) * 3 * nv);
  double* v1 = malloc(sizeof(double) * 3 * nv);
  if (!ev || !v1) {
    if (!evals) free(ev);
    free(v1);
    return CTO_ERR_OOM;
  }
  cto_eig_field(S, nv, ev, v1);
  rc = cto_angles_field3(v1, ev, dims, lo, n, center, axis, spacing, centres, mask, fill, vout, ha, ia, fa);
  if (!evals) free(ev);
  free(v1);
  return rc;
}

int cto_pipeline(const uint16_t* vol, const int64_t dims[3], const int64_t lo[3], const int64_t n[3], double sigma,
                 double rho, double truncate, const double center[3], const double axis[3], const uint8_t* mask,
                 double fill, double* S, double* evals, double* vout, double* ha, double* ia, double* fa) {
  const double one[3] = {1.0, 1.0, 1.0};
  return cto_pipeline3(vol, dims, lo, n, sigma, rho, truncate, one, center, axis, NULL, mask, fill, S, evals, vout,
                       ha, ia, fa);
}

/* Threads OpenMP will use (1 when built without OpenMP). */
int cto_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Set the threads later calls use (the benchmark's 1-core figure); no-op
   without OpenMP. */
void cto_set_num_threads(int n) {
#ifdef _OPENMP
  extern void omp_set_num_threads(int);
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}
