/*
 * contacts_oracle.c -- plain FP64 CPU oracle of the order in which native
 * contacts form along a path and of the path similarity of the variational
 * pathway scheme (arXiv:1405.6104, Sec. "Results", folding-mechanism
 * matrix M and path similarity s(k, k'), after Camilloni et al. 2011).
 *
 * TEST INFRASTRUCTURE ONLY, like vpath_oracle.c (linked into the same
 * stand-alone library; nothing here is shared with the CUDA library).
 *
 * Definitions (with the readings the paper leaves open):
 *   - a contact (i, j) between CV atoms with j - i > min_sep is "formed"
 *     when its contact value C(r) = (1 - (r/r0)^6)/(1 - (r/r0)^10) exceeds
 *     1/2.  With s = (r/r0)^2, C > 1/2  <=>  1 + s + s^2 > s^3 + s^4
 *     <=>  p(s) = s^4 + s^3 - s^2 - s - 1 < 0, which is how it is decided
 *     (no division by the removable singularity at s = 1);
 *   - native contacts: the contacts formed in the native structure
 *     (Euclidean distances);
 *   - formation time t_i of a native contact along a path: the first time
 *     from which it stays formed to the end of the path; -1 when it is not
 *     formed at the end (it orders after every formed contact);
 *   - M_ij = 1 if t_i < t_j, 0 if t_i > t_j, 1/2 if t_i = t_j, and
 *     s(k, k') = (1 / (Nc (Nc - 1))) sum_{i != j} [M_ij(k) = M_ij(k')].
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

static double min_image_c(double d, double L) { return d - L * nearbyint(d / L); }

static int formed(double r2, double r0) {
  double s = r2 / (r0 * r0);
  double p = (((s + 1.0) * s - 1.0) * s - 1.0) * s - 1.0;
  return p < 0.0;
}

/* Native contacts (i < j, j - i > min_sep, formed in the native structure),
 * in order of i then j; returns their number (pairs beyond cap dropped). */
int64_t or_native_contacts(const double *native, int32_t n_cv, double r0, int32_t min_sep, int32_t *pairs,
                           int64_t cap) {
  int64_t n = 0;
  for (int32_t i = 0; i < n_cv; ++i)
    for (int32_t j = i + min_sep + 1; j < n_cv; ++j) {
      double dx = native[3 * j] - native[3 * i];
      double dy = native[3 * j + 1] - native[3 * i + 1];
      double dz = native[3 * j + 2] - native[3 * i + 2];
      if (formed(dx * dx + dy * dy + dz * dz, r0)) {
        if (n < cap) { pairs[2 * n] = i; pairs[2 * n + 1] = j; }
        ++n;
      }
    }
  return n;
}

/* Formation times of the given contacts along frames [n_frames][n_cv][3]
 * taken at the step numbers steps[]; positions in a cubic box of side box
 * (minimum image). */
void or_contact_times(const double *frames, const int64_t *steps, int32_t n_frames, int32_t n_cv, double box,
                      double r0, const int32_t *pairs, int64_t n_c, int64_t *t) {
  for (int64_t c = 0; c < n_c; ++c) t[c] = -1;
  for (int32_t f = 0; f < n_frames; ++f) {
    const double *X = frames + (size_t)f * 3 * (size_t)n_cv;
    for (int64_t c = 0; c < n_c; ++c) {
      int i = pairs[2 * c], j = pairs[2 * c + 1];
      double dx = min_image_c(X[3 * j] - X[3 * i], box);
      double dy = min_image_c(X[3 * j + 1] - X[3 * i + 1], box);
      double dz = min_image_c(X[3 * j + 2] - X[3 * i + 2], box);
      if (formed(dx * dx + dy * dy + dz * dz, r0)) {
        if (t[c] < 0) t[c] = steps[f];
      } else {
        t[c] = -1;
      }
    }
  }
}

static double order_entry(int64_t ti, int64_t tj) {
  /* an unformed contact (-1) forms "at infinity" */
  double a = ti < 0 ? INFINITY : (double)ti, b = tj < 0 ? INFINITY : (double)tj;
  if (a < b) return 1.0;
  if (a > b) return 0.0;
  return 0.5;
}

/* Path similarity of two paths from their formation times. */
double or_path_similarity(const int64_t *ta, const int64_t *tb, int64_t n_c) {
  if (n_c < 2) return 1.0;
  int64_t same = 0;
  for (int64_t i = 0; i < n_c; ++i)
    for (int64_t j = 0; j < n_c; ++j)
      if (i != j && order_entry(ta[i], ta[j]) == order_entry(tb[i], tb[j])) ++same;
  return (double)same / ((double)n_c * (double)(n_c - 1));
}
