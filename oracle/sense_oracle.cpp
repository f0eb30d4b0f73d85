// FP64 CPU oracle for Cartesian multi-coil SENSE (TEST INFRASTRUCTURE ONLY).
//
// This file is the plain, slow, obviously-correct reference that the CUDA
// library is checked against.  It shares no code, header, table or constant
// with the GPU path.  Only tests, the smoke check and the CPU-baseline leg of
// the benchmark may load it; the product library never does.
//
// What it computes (arXiv 1807.11830, Sec. IV-A, Eq. 1, and the CG-SENSE
// extension built on it):
//   * unitary DFT, direct O(n^2) form and a recursive mixed-radix FFT;
//   * encoding operator  E : y[f][c][l][:] = (F2 (S_c . x_f))[lines[f][l]][:]
//   * adjoint          E^H : x_f = sum_c conj(S_c) . F2^H(Z_f y_{f,c})
//     which, with every line sampled, is Eq. 1: M = sum_i S_i^* F^{-1}(Y_i);
//   * normal operator E^H E, computed literally as adjoint(forward(x));
//   * a separate column-wise ("1D collapsed") normal operator used only to
//     pin the algebra the GPU path relies on;
//   * Hestenes-Stiefel conjugate gradients on E^H E x = E^H y, per frame;
//   * root-sum-of-squares coil combine (Sec. IV-B);
//   * IEEE binary32 -> bfloat16 round-to-nearest-even from the format's
//     definition.
//
// Conventions (readings of the paper where it is silent):
//   * F is unitary: forward kernel exp(-2 pi i jk/n)/sqrt(n), inverse the
//     conjugate with the same scale (Eq. 1 writes F^{-1} without a scale).
//   * DC sits at index 0 (no fftshift) unless an entry point's `centred` is
//     1: then every transform is the centred one, DC and the image centre at
//     index floor(n/2) along each axis, defined as fftshift . F . ifftshift
//     (fftshift rotates by floor(n/2), ifftshift back), and the line indices
//     address that centred k-space.  y (slow index, rows) is the masked
//     phase-encode direction; x (fast index) is the fully sampled readout.
//   * lines[f][0..L) is strictly increasing inside [0, ny).
//   * complex arrays are interleaved (re, im) doubles, row-major:
//       x [F][ny][nx], S [C][ny][nx], y [F][C][L][nx], lines [F][L].
//
// Parity pins for every function live in tests/test_oracle_pins.py.

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using cd = std::complex<double>;
const double kTwoPi = 6.283185307179586476925286766559;

// exp(dir * 2 pi i * m / n) with m reduced modulo n first, so the angle
// never grows with the product of indices.
cd unit_root(long long m, long long n, int dir) {
  long long r = m % n;
  if (r < 0) r += n;
  double ang = dir * kTwoPi * (double)r / (double)n;
  return cd(std::cos(ang), std::sin(ang));
}

// Direct DFT, unnormalised: X[k] = sum_j x[j*stride] w^{jk}, w = e^{dir 2 pi i/n}.
void dft_direct(int n, int dir, const cd* in, long stride, cd* out) {
  for (int k = 0; k < n; ++k) {
    cd acc(0.0, 0.0);
    for (int j = 0; j < n; ++j) acc += in[(long)j * stride] * unit_root((long long)j * k, n, dir);
    out[k] = acc;
  }
}

int smallest_factor(int n) {
  if (n % 2 == 0) return 2;
  if (n % 3 == 0) return 3;
  if (n % 5 == 0) return 5;
  return n;  // anything else is handled by the direct DFT
}

// Recursive decimation-in-time Cooley-Tukey, unnormalised.  With n = p*m,
// sample j = p*a + r (r in [0,p)) feeds sub-transform r of length m; output
//   X[k + m s] = sum_r w_n^{r (k + m s)} T_r[k].
void fft_rec(int n, int dir, const cd* in, long stride, cd* out) {
  if (n == 1) { out[0] = in[0]; return; }
  int p = smallest_factor(n);
  if (p == n) { dft_direct(n, dir, in, stride, out); return; }
  int m = n / p;
  std::vector<cd> sub((size_t)n);
  for (int r = 0; r < p; ++r) fft_rec(m, dir, in + (long)r * stride, stride * p, sub.data() + (size_t)r * m);
  for (int k = 0; k < m; ++k) {
    for (int s = 0; s < p; ++s) {
      long long kk = k + (long long)m * s;
      cd acc(0.0, 0.0);
      for (int r = 0; r < p; ++r) acc += sub[(size_t)r * m + k] * unit_root((long long)r * kk, n, dir);
      out[kk] = acc;
    }
  }
}

// Unitary 1D transform of a strided sequence, written back in place.
void fft1_strided(int n, int dir, cd* data, long stride, std::vector<cd>& tmp_in, std::vector<cd>& tmp_out) {
  tmp_in.resize(n);
  tmp_out.resize(n);
  for (int j = 0; j < n; ++j) tmp_in[j] = data[(long)j * stride];
  fft_rec(n, dir, tmp_in.data(), 1, tmp_out.data());
  double s = 1.0 / std::sqrt((double)n);
  for (int j = 0; j < n; ++j) data[(long)j * stride] = tmp_out[j] * s;
}

// Rotate v[0], v[stride], ..., v[(n-1) stride] so that element i moves to
// (i + shift) mod n.
void rotate_strided(int n, cd* v, long stride, int shift) {
  std::vector<cd> t((size_t)n);
  for (int i = 0; i < n; ++i) t[((i + shift) % n + n) % n] = v[(long)i * stride];
  for (int i = 0; i < n; ++i) v[(long)i * stride] = t[i];
}

// Unitary transform of one strided sequence; centred: fftshift . F . ifftshift.
void fft1_conv(int n, int dir, cd* v, long stride, bool centred, std::vector<cd>& a, std::vector<cd>& b) {
  if (centred) rotate_strided(n, v, stride, -(n / 2));  // ifftshift
  fft1_strided(n, dir, v, stride, a, b);
  if (centred) rotate_strided(n, v, stride, n / 2);  // fftshift
}

// Unitary 2D transform F2 = F_y F_x of one [ny][nx] image, in place.
void fft2_inplace(int ny, int nx, int dir, cd* img, bool centred = false) {
  std::vector<cd> a, b;
  for (int r = 0; r < ny; ++r) fft1_conv(nx, dir, img + (long)r * nx, 1, centred, a, b);
  for (int c = 0; c < nx; ++c) fft1_conv(ny, dir, img + c, nx, centred, a, b);
}

bool lines_ok(int ny, int L, const int* ln) {
  for (int l = 0; l < L; ++l) {
    if (ln[l] < 0 || ln[l] >= ny) return false;
    if (l > 0 && ln[l] <= ln[l - 1]) return false;
  }
  return true;
}

bool all_lines_ok(int F, int ny, int L, const int* lines) {
  for (int f = 0; f < F; ++f)
    if (!lines_ok(ny, L, lines + (long)f * L)) return false;
  return true;
}

// E for one frame: y_f[c][l][:] = F2(S_c . x_f)[ln[l]][:].
void forward_frame(int C, int ny, int nx, int L, const cd* xf, const cd* S, const int* ln, cd* yf, bool centred) {
  long npix = (long)ny * nx;
  std::vector<cd> t((size_t)npix);
  for (int c = 0; c < C; ++c) {
    const cd* Sc = S + c * npix;
    for (long i = 0; i < npix; ++i) t[i] = Sc[i] * xf[i];
    fft2_inplace(ny, nx, -1, t.data(), centred);
    for (int l = 0; l < L; ++l)
      for (int k = 0; k < nx; ++k) yf[((long)c * L + l) * nx + k] = t[(long)ln[l] * nx + k];
  }
}

// E^H for one frame: x_f = sum_c conj(S_c) . F2^H(Z y_{f,c}), Z the zero-fill.
void adjoint_frame(int C, int ny, int nx, int L, const cd* yf, const cd* S, const int* ln, cd* xf, bool centred) {
  long npix = (long)ny * nx;
  std::vector<cd> z((size_t)npix);
  for (long i = 0; i < npix; ++i) xf[i] = 0.0;
  for (int c = 0; c < C; ++c) {
    for (long i = 0; i < npix; ++i) z[i] = 0.0;
    for (int l = 0; l < L; ++l)
      for (int k = 0; k < nx; ++k) z[(long)ln[l] * nx + k] = yf[((long)c * L + l) * nx + k];
    fft2_inplace(ny, nx, +1, z.data(), centred);
    const cd* Sc = S + c * npix;
    for (long i = 0; i < npix; ++i) xf[i] += std::conj(Sc[i]) * z[i];
  }
}

// E^H E for one frame, literally adjoint(forward(.)).
void normal_frame(int C, int ny, int nx, int L, const cd* xf, const cd* S, const int* ln, cd* of, bool centred) {
  std::vector<cd> y((size_t)C * L * nx);
  forward_frame(C, ny, nx, L, xf, S, ln, y.data(), centred);
  adjoint_frame(C, ny, nx, L, y.data(), S, ln, of, centred);
}

// Re <a, b> = Re sum conj(a) b, sequential sum.
double re_dot(long n, const cd* a, const cd* b) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += a[i].real() * b[i].real() + a[i].imag() * b[i].imag();
  return s;
}

// CG over all frames at once on
//   (E^H E + lambda I + lambda_t L) x = E^H y,
// L the cyclic second difference across frames, (L x)_f = 2 x_f - x_{f-1} -
// x_{f+1} with frame indices modulo F: the normal equations of
// ||E x - y||^2 + lambda ||x||^2 + lambda_t sum_f ||x_f - x_{f-1}||^2 for a
// cyclic (cine) series.  One set of scalars for the stacked vector; every
// frame reports the same iterations, residual and status.
void cg_coupled(int F, int C, int ny, int nx, int L, const cd* yc, const cd* Sc, const int* lines, int max_iter,
                double tol, bool centred, double lambda, double lambda_t, cd* x, int* iters, double* resid,
                int* status) {
  const long npix = (long)ny * nx, n = (long)F * npix;
  std::vector<cd> r((size_t)n), p((size_t)n), q((size_t)n);
  for (int f = 0; f < F; ++f)
    adjoint_frame(C, ny, nx, L, yc + (long)f * C * L * nx, Sc, lines + (long)f * L, r.data() + f * npix, centred);
  for (long i = 0; i < n; ++i) { x[i] = 0.0; p[i] = r[i]; }
  double rho = re_dot(n, r.data(), r.data());
  const double rho0 = rho;
  int it = 0;
  int st = rho0 == 0.0 ? 1 : 0;  // converged / running
  while (st == 0 && it < max_iter) {
    for (int f = 0; f < F; ++f) {
      cd* qf = q.data() + f * npix;
      const cd* pf = p.data() + f * npix;
      const cd* pm = p.data() + (long)((f + F - 1) % F) * npix;
      const cd* pn = p.data() + (long)((f + 1) % F) * npix;
      normal_frame(C, ny, nx, L, pf, Sc, lines + (long)f * L, qf, centred);
      for (long i = 0; i < npix; ++i) qf[i] += lambda * pf[i] + lambda_t * (2.0 * pf[i] - pm[i] - pn[i]);
    }
    const double pq = re_dot(n, p.data(), q.data());
    if (!(pq > 0.0)) { st = 3; break; }
    const double alpha = rho / pq;
    for (long i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    const double rho_new = re_dot(n, r.data(), r.data());
    ++it;
    if (rho_new == 0.0 || (tol > 0.0 && std::sqrt(rho_new / rho0) <= tol)) {
      rho = rho_new;
      st = 1;
      break;
    }
    const double beta = rho_new / rho;
    for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    rho = rho_new;
  }
  if (st == 0) st = 2;
  for (int f = 0; f < F; ++f) {
    iters[f] = it;
    resid[f] = rho0 > 0.0 ? std::sqrt(rho / rho0) : 0.0;
    status[f] = st;
  }
}

}  // namespace

extern "C" {

// Status codes of the oracle entry points.
enum { ORC_OK = 0, ORC_EINVAL = 1 };

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

// Unitary direct DFT of length n (dir -1 forward, +1 inverse).
int orc_dft(int n, int dir, const double* in, double* out) {
  if (n <= 0 || (dir != 1 && dir != -1)) return ORC_EINVAL;
  const cd* a = reinterpret_cast<const cd*>(in);
  cd* b = reinterpret_cast<cd*>(out);
  std::vector<cd> tmp((size_t)n);
  dft_direct(n, dir, a, 1, tmp.data());
  double s = 1.0 / std::sqrt((double)n);
  for (int k = 0; k < n; ++k) b[k] = tmp[k] * s;
  return ORC_OK;
}

// Unitary recursive mixed-radix FFT of length n.
int orc_fft(int n, int dir, const double* in, double* out) {
  if (n <= 0 || (dir != 1 && dir != -1)) return ORC_EINVAL;
  const cd* a = reinterpret_cast<const cd*>(in);
  cd* b = reinterpret_cast<cd*>(out);
  std::vector<cd> tmp((size_t)n);
  fft_rec(n, dir, a, 1, tmp.data());
  double s = 1.0 / std::sqrt((double)n);
  for (int k = 0; k < n; ++k) b[k] = tmp[k] * s;
  return ORC_OK;
}

// Unitary 2D transform F2 = F_y F_x of `count` stacked [ny][nx] images.
int orc_fft2(int count, int ny, int nx, int dir, const double* in, double* out, int centred) {
  if (count < 0 || ny <= 0 || nx <= 0 || (dir != 1 && dir != -1)) return ORC_EINVAL;
  long npix = (long)ny * nx;
  if (out != in) std::memcpy(out, in, sizeof(double) * 2 * npix * count);
  cd* b = reinterpret_cast<cd*>(out);
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < count; ++i) fft2_inplace(ny, nx, dir, b + i * npix, centred != 0);
  return ORC_OK;
}

int orc_forward(int F, int C, int ny, int nx, int L, const double* x, const double* S, const int* lines,
                double* y, int centred) {
  if (F < 0 || C <= 0 || ny <= 0 || nx <= 0 || L < 0 || L > ny) return ORC_EINVAL;
  if (!all_lines_ok(F, ny, L, lines)) return ORC_EINVAL;
  long npix = (long)ny * nx;
  const cd* xc = reinterpret_cast<const cd*>(x);
  const cd* Sc = reinterpret_cast<const cd*>(S);
  cd* yc = reinterpret_cast<cd*>(y);
#pragma omp parallel for schedule(dynamic)
  for (int f = 0; f < F; ++f)
    forward_frame(C, ny, nx, L, xc + f * npix, Sc, lines + (long)f * L, yc + (long)f * C * L * nx, centred != 0);
  return ORC_OK;
}

int orc_adjoint(int F, int C, int ny, int nx, int L, const double* y, const double* S, const int* lines,
                double* x, int centred) {
  if (F < 0 || C <= 0 || ny <= 0 || nx <= 0 || L < 0 || L > ny) return ORC_EINVAL;
  if (!all_lines_ok(F, ny, L, lines)) return ORC_EINVAL;
  long npix = (long)ny * nx;
  const cd* yc = reinterpret_cast<const cd*>(y);
  const cd* Sc = reinterpret_cast<const cd*>(S);
  cd* xc = reinterpret_cast<cd*>(x);
#pragma omp parallel for schedule(dynamic)
  for (int f = 0; f < F; ++f)
    adjoint_frame(C, ny, nx, L, yc + (long)f * C * L * nx, Sc, lines + (long)f * L, xc + f * npix, centred != 0);
  return ORC_OK;
}

// Literal E^H(E x).
int orc_normal(int F, int C, int ny, int nx, int L, const double* x, const double* S, const int* lines,
               double* out, int centred) {
  if (F < 0 || C <= 0 || ny <= 0 || nx <= 0 || L < 0 || L > ny) return ORC_EINVAL;
  if (!all_lines_ok(F, ny, L, lines)) return ORC_EINVAL;
  long npix = (long)ny * nx;
  const cd* xc = reinterpret_cast<const cd*>(x);
  const cd* Sc = reinterpret_cast<const cd*>(S);
  cd* oc = reinterpret_cast<cd*>(out);
#pragma omp parallel for schedule(dynamic)
  for (int f = 0; f < F; ++f)
    normal_frame(C, ny, nx, L, xc + f * npix, Sc, lines + (long)f * L, oc + f * npix, centred != 0);
  return ORC_OK;
}

// Column-wise form of the normal operator:
//   out_f[:, j] = sum_c conj(S_c[:, j]) . F_y^H M_f F_y (S_c[:, j] . x_f[:, j])
// for every column j.  It is a second, independent route to E^H E (the x
// transform cancels because the mask acts on rows only); it exists so a test
// can pin the identity the GPU kernels are built on.
int orc_normal_collapsed(int F, int C, int ny, int nx, int L, const double* x, const double* S,
                         const int* lines, double* out) {
  if (F < 0 || C <= 0 || ny <= 0 || nx <= 0 || L < 0 || L > ny) return ORC_EINVAL;
  if (!all_lines_ok(F, ny, L, lines)) return ORC_EINVAL;
  long npix = (long)ny * nx;
  const cd* xc = reinterpret_cast<const cd*>(x);
  const cd* Sc = reinterpret_cast<const cd*>(S);
  cd* oc = reinterpret_cast<cd*>(out);
#pragma omp parallel for schedule(dynamic)
  for (int f = 0; f < F; ++f) {
    const int* ln = lines + (long)f * L;
    std::vector<char> sampled((size_t)ny, 0);
    for (int l = 0; l < L; ++l) sampled[ln[l]] = 1;
    std::vector<cd> col((size_t)ny), a, b;
    const cd* xf = xc + f * npix;
    cd* of = oc + f * npix;
    for (long i = 0; i < npix; ++i) of[i] = 0.0;
    for (int j = 0; j < nx; ++j) {
      for (int c = 0; c < C; ++c) {
        const cd* S_c = Sc + c * npix;
        for (int r = 0; r < ny; ++r) col[r] = S_c[(long)r * nx + j] * xf[(long)r * nx + j];
        fft1_strided(ny, -1, col.data(), 1, a, b);
        for (int r = 0; r < ny; ++r)
          if (!sampled[r]) col[r] = 0.0;
        fft1_strided(ny, +1, col.data(), 1, a, b);
        for (int r = 0; r < ny; ++r) of[(long)r * nx + j] += std::conj(S_c[(long)r * nx + j]) * col[r];
      }
    }
  }
  return ORC_OK;
}

// Per-frame CG status values written to status[f].
enum { ORC_CG_RUNNING = 0, ORC_CG_CONVERGED = 1, ORC_CG_MAXITER = 2, ORC_CG_BREAKDOWN = 3 };

// Hestenes-Stiefel CG on (E^H E + lambda I) x = E^H y, independently for
// every frame (lambda >= 0 is Tikhonov regularisation; 0 gives CG-SENSE);
// lambda_t > 0 adds the temporal term and couples the frames (cg_coupled):
//   b = E^H y; x0 = 0; r0 = b; p0 = r0; rho0 = <r0, r0>
//   for k = 0 .. max_iter-1:
//     q = E^H E p + lambda p;  alpha = rho_k / Re<p, q>
//     x += alpha p;  r -= alpha q;  rho_{k+1} = <r, r>
//     stop if rho_{k+1} == 0, or tol > 0 and sqrt(rho_{k+1}/rho0) <= tol
//     beta = rho_{k+1} / rho_k;  p = r + beta p
// Breakdown: if Re<p,q> is not > 0 (zero, negative or NaN) the frame stops
// before updating x and is marked ORC_CG_BREAKDOWN.  A frame with b == 0
// returns x = 0 after zero iterations.
// Outputs: x [F][ny][nx]; iters[f] = iterations applied; resid[f] =
// sqrt(rho/rho0) at exit (0 when rho0 == 0); status[f] as above.
int orc_cg(int F, int C, int ny, int nx, int L, const double* y, const double* S, const int* lines, int max_iter,
           double tol, double* x, int* iters, double* resid, int* status, int centred, double lambda,
           double lambda_t) {
  if (F < 0 || C <= 0 || ny <= 0 || nx <= 0 || L < 0 || L > ny || max_iter < 0 || !(tol >= 0.0) ||
      !(lambda >= 0.0) || !(lambda_t >= 0.0))
    return ORC_EINVAL;
  if (!all_lines_ok(F, ny, L, lines)) return ORC_EINVAL;
  long npix = (long)ny * nx;
  const cd* yc = reinterpret_cast<const cd*>(y);
  const cd* Sc = reinterpret_cast<const cd*>(S);
  cd* xc = reinterpret_cast<cd*>(x);
  if (lambda_t > 0.0) {  // frames coupled: one CG over the series
    cg_coupled(F, C, ny, nx, L, yc, Sc, lines, max_iter, tol, centred != 0, lambda, lambda_t, xc, iters, resid,
               status);
    return ORC_OK;
  }
#pragma omp parallel for schedule(dynamic)
  for (int f = 0; f < F; ++f) {
    const int* ln = lines + (long)f * L;
    cd* xf = xc + f * npix;
    std::vector<cd> r((size_t)npix), p((size_t)npix), q((size_t)npix);
    adjoint_frame(C, ny, nx, L, yc + (long)f * C * L * nx, Sc, ln, r.data(), centred != 0);
    for (long i = 0; i < npix; ++i) { xf[i] = 0.0; p[i] = r[i]; }
    double rho = re_dot(npix, r.data(), r.data());
    double rho0 = rho;
    int it = 0;
    int st = ORC_CG_RUNNING;
    if (rho0 == 0.0) st = ORC_CG_CONVERGED;
    while (st == ORC_CG_RUNNING && it < max_iter) {
      normal_frame(C, ny, nx, L, p.data(), Sc, ln, q.data(), centred != 0);
      for (long i = 0; i < npix; ++i) q[i] += lambda * p[i];
      double pq = re_dot(npix, p.data(), q.data());
      if (!(pq > 0.0)) { st = ORC_CG_BREAKDOWN; break; }
      double alpha = rho / pq;
      for (long i = 0; i < npix; ++i) {
        xf[i] += alpha * p[i];
        r[i] -= alpha * q[i];
      }
      double rho_new = re_dot(npix, r.data(), r.data());
      ++it;
      if (rho_new == 0.0 || (tol > 0.0 && std::sqrt(rho_new / rho0) <= tol)) {
        rho = rho_new;
        st = ORC_CG_CONVERGED;
        break;
      }
      double beta = rho_new / rho;
      for (long i = 0; i < npix; ++i) p[i] = r[i] + beta * p[i];
      rho = rho_new;
    }
    if (st == ORC_CG_RUNNING) st = ORC_CG_MAXITER;
    iters[f] = it;
    resid[f] = rho0 > 0.0 ? std::sqrt(rho / rho0) : 0.0;
    status[f] = st;
  }
  return ORC_OK;
}

// Root sum of squares (Sec. IV-B): per frame and pixel,
//   out[f][i] = sqrt(sum_c |F2^H(Z y_{f,c})[i]|^2)
// with y [F][C][L][nx] and the same line convention as orc_adjoint.
int orc_rss(int F, int C, int ny, int nx, int L, const double* y, const int* lines, double* out, int centred) {
  if (F < 0 || C <= 0 || ny <= 0 || nx <= 0 || L < 0 || L > ny) return ORC_EINVAL;
  if (!all_lines_ok(F, ny, L, lines)) return ORC_EINVAL;
  long npix = (long)ny * nx;
  const cd* yc = reinterpret_cast<const cd*>(y);
#pragma omp parallel for schedule(dynamic)
  for (int f = 0; f < F; ++f) {
    const int* ln = lines + (long)f * L;
    std::vector<cd> z((size_t)npix);
    std::vector<double> acc((size_t)npix, 0.0);
    for (int c = 0; c < C; ++c) {
      for (long i = 0; i < npix; ++i) z[i] = 0.0;
      const cd* yfc = yc + ((long)f * C + c) * L * nx;
      for (int l = 0; l < L; ++l)
        for (int k = 0; k < nx; ++k) z[(long)ln[l] * nx + k] = yfc[(long)l * nx + k];
      fft2_inplace(ny, nx, +1, z.data(), centred != 0);
      for (long i = 0; i < npix; ++i) acc[i] += std::norm(z[i]);
    }
    for (long i = 0; i < npix; ++i) out[f * npix + i] = std::sqrt(acc[i]);
  }
  return ORC_OK;
}

// binary32 -> bfloat16, round to nearest, ties to even, written from the
// formats' definitions: bfloat16 keeps the sign, the 8 exponent bits and the
// top 7 fraction bits of binary32.  The 16 dropped bits decide the rounding:
// above half an ulp round up, below round down, exactly half round to the
// neighbour whose last kept bit is 0.  A carry out of the fraction moves into
// the exponent, which is how values round up into the next binade or to
// infinity.  NaNs stay NaN (quiet bit set).
void orc_bf16_rne(long n, const float* in, uint16_t* out) {
  for (long i = 0; i < n; ++i) {
    uint32_t u;
    std::memcpy(&u, &in[i], 4);
    uint32_t exp_bits = (u >> 23) & 0xFFu;
    uint32_t frac_bits = u & 0x7FFFFFu;
    if (exp_bits == 0xFFu && frac_bits != 0) {  // NaN
      out[i] = (uint16_t)((u >> 16) | 0x0040u);
      continue;
    }
    uint32_t kept = u >> 16;
    uint32_t dropped = u & 0xFFFFu;
    bool up = dropped > 0x8000u || (dropped == 0x8000u && (kept & 1u));
    if (up) kept += 1u;
    out[i] = (uint16_t)kept;
  }
}

}  // extern "C"
