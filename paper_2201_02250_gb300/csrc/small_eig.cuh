// Dense real non-symmetric eigensolver for the small Rayleigh-Ritz matrices of
// the local eigenproblems (order <= a few hundred).  Householder reduction to
// upper Hessenberg form, Francis implicit double-shift QR iteration to real
// Schur form (Golub & Van Loan, Matrix Computations, Sections 7.4-7.5),
// eigenvectors by back-substitution on the quasi-triangular factor.
//
// The routines run on a "team": on the GPU the threads of one CTA (lane = thread
// id, size = block size, sync = __syncthreads), on the host a single thread
// (lane 0, size 1, no sync).
// The matrix is row-major with leading dimension ld and lives in memory the
// whole team can address (shared memory on the GPU).
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define SE_HD __host__ __device__
#else
#define SE_HD
#endif

namespace a2ls {
namespace se {

struct Team {
  int lane, size;
  SE_HD void sync() const {
#ifdef __CUDA_ARCH__
    __syncthreads();
#endif
  }
};

// Scalar helpers of the arithmetic R the routines run in (double here; other arithmetics provide
// their own overloads of se_abs, se_sqrt and se_dbl next to their type and specialise SeEps).
SE_HD inline double se_abs(double x) { return fabs(x); }
SE_HD inline double se_sqrt(double x) { return sqrt(x); }
SE_HD inline double se_dbl(double x) { return x; }
// acc += a * b in the dot products, and the value of an accumulator (an arithmetic with a cheaper
// unnormalised multiply-add overloads both)
SE_HD inline void se_mac(double& acc, double a, double b) { acc += a * b; }
SE_HD inline double se_fin(double a) { return a; }
template <class R> struct SeEps {
  static constexpr double v = 2.220446049250313e-16;  // machine epsilon of R
  static constexpr double big = 1e100;                // rescaling threshold of the back substitution
};

// Whether the Francis iteration forms the next bulge reflector during the right update (one thread,
// from a snapshot) rather than with every thread after it.  Measured on GB300: faster in FP64
// (Rayleigh-Ritz 178 -> 147 ms per 512x512 setup), slower in double-float (28.7 -> 30.3 ms), whose
// longer reflector arithmetic on one thread outlasts the right update.
template <class R> struct SeEarlyReflector { static constexpr bool value = true; };

template <class R>
SE_HD inline R sgn(R a, R b) { return b >= R(0.0) ? se_abs(a) : -se_abs(a); }

// Reduce H (m x m) to upper Hessenberg form, accumulating the orthogonal factor in Q (Q <- Q P).
// v: scratch of m values.  Each reflector takes two phases of the team: the left update (one column
// per thread) together with the first rows of Q, then the right update of H (one row per thread)
// together with the remaining rows of Q (with 128 threads and m <= 85 no thread holds more than one
// item per phase).
template <class R>
SE_HD inline void hessenberg(R* H, int ld, R* Q, int ldq, int m, R* v, const Team& t) {
  for (int k = 0; k + 2 < m; ++k) {
    // Householder vector for x = H[k+1.., k]
    R nrm2 = 0.0;
    for (int r = k + 1; r < m; ++r) se_mac(nrm2, H[r * ld + k], H[r * ld + k]);
    nrm2 = se_fin(nrm2);
    R nrm = se_sqrt(nrm2);
    if (nrm == 0.0) continue;
    R x0 = H[(k + 1) * ld + k];
    R alpha = -sgn(nrm, x0);
    // v = x - alpha e1, scaled so that P = I - 2 v v^T / (v^T v); v^T v = 2 nrm |x0 - alpha|
    R vtv = nrm2 - x0 * x0 + (x0 - alpha) * (x0 - alpha);
    if (vtv == 0.0) continue;
    t.sync();
    for (int r = k + 1 + t.lane; r < m; r += t.size) v[r] = (r == k + 1) ? (x0 - alpha) : H[r * ld + k];
    t.sync();
    const R beta = 2.0 / vtv;
    const int ncol = m - k;                                  // left update: columns k..m-1
    const int qa = (t.size > ncol) ? ((t.size - ncol < m) ? t.size - ncol : m) : 0;  // Q rows in phase 1
    for (int idx = t.lane; idx < ncol + qa; idx += t.size) {
      if (idx < ncol) {
        const int c = k + idx;
        R d = 0.0;
        for (int r = k + 1; r < m; ++r) se_mac(d, v[r], H[r * ld + c]);
        d = se_fin(d) * beta;
        for (int r = k + 1; r < m; ++r) H[r * ld + c] -= d * v[r];
      } else {
        const int r = idx - ncol;
        R e = 0.0;
        for (int c = k + 1; c < m; ++c) se_mac(e, Q[r * ldq + c], v[c]);
        e = se_fin(e) * beta;
        for (int c = k + 1; c < m; ++c) Q[r * ldq + c] -= e * v[c];
      }
    }
    t.sync();
    // right: all rows of H, columns k+1..; the remaining rows of Q
    for (int idx = t.lane; idx < m + (m - qa); idx += t.size) {
      if (idx < m) {
        const int r = idx;
        R d = 0.0;
        for (int c = k + 1; c < m; ++c) se_mac(d, H[r * ld + c], v[c]);
        d = se_fin(d) * beta;
        for (int c = k + 1; c < m; ++c) H[r * ld + c] -= d * v[c];
      } else {
        const int r = qa + idx - m;
        R e = 0.0;
        for (int c = k + 1; c < m; ++c) se_mac(e, Q[r * ldq + c], v[c]);
        e = se_fin(e) * beta;
        for (int c = k + 1; c < m; ++c) Q[r * ldq + c] -= e * v[c];
      }
    }
    t.sync();
    if (t.lane == 0) {
      H[(k + 1) * ld + k] = alpha;
      for (int r = k + 2; r < m; ++r) H[r * ld + k] = 0.0;
    }
    t.sync();
  }
}

// Apply a 3-element (or 2-element when nv == 2) reflector I - beta u u^T with u = (1, u1, u2)
// to rows k..k+nv-1 of H from the left (columns c0..m-1) and to columns k..k+nv-1 from the
// right (rows 0..r1) and to Q's columns.
template <class R>
SE_HD inline void apply_reflector(R* H, int ld, R* Q, int ldq, int m, int k, int nv, R u1, R u2, R beta,
                                  int c0, int r1, const Team& t) {
  for (int c = c0 + t.lane; c < m; c += t.size) {
    R d = H[k * ld + c] + u1 * H[(k + 1) * ld + c] + (nv == 3 ? u2 * H[(k + 2) * ld + c] : 0.0);
    d *= beta;
    H[k * ld + c] -= d;
    H[(k + 1) * ld + c] -= d * u1;
    if (nv == 3) H[(k + 2) * ld + c] -= d * u2;
  }
  t.sync();
  for (int r = t.lane; r <= r1; r += t.size) {
    R d = H[r * ld + k] + u1 * H[r * ld + k + 1] + (nv == 3 ? u2 * H[r * ld + k + 2] : 0.0);
    d *= beta;
    H[r * ld + k] -= d;
    H[r * ld + k + 1] -= d * u1;
    if (nv == 3) H[r * ld + k + 2] -= d * u2;
  }
  for (int r = t.lane; r < m; r += t.size) {
    R d = Q[r * ldq + k] + u1 * Q[r * ldq + k + 1] + (nv == 3 ? u2 * Q[r * ldq + k + 2] : 0.0);
    d *= beta;
    Q[r * ldq + k] -= d;
    Q[r * ldq + k + 1] -= d * u1;
    if (nv == 3) Q[r * ldq + k + 2] -= d * u2;
  }
  t.sync();
}

// Householder reflector mapping (x, y, z) to (alpha, 0, 0): returns alpha, beta and u = (1, u1, u2).
// With v = (v0, y, z), v0 = x - alpha, v^T v = 2 |alpha| |v0|, so beta = 2 v0^2 / v^T v = v0 / (-alpha).
template <class R>
SE_HD inline bool make_reflector(R x, R y, R z, R& u1, R& u2, R& beta, R& alpha) {
  R nrm = se_sqrt(x * x + y * y + z * z);
  if (nrm == 0.0) return false;
  alpha = -sgn(nrm, x);
  R v0 = x - alpha;
  if (v0 == 0.0) return false;
  const R iv = R(1.0) / v0;
  u1 = y * iv;
  u2 = z * iv;
  beta = v0 / (-alpha);
  return true;
}

// Make a 2x2 diagonal block with real eigenvalues upper triangular by a rotation (rows/cols p, p+1).
template <class R>
SE_HD inline void split_2x2(R* H, int ld, R* Q, int ldq, int m, int p, const Team& t) {
  t.sync();
  R a = H[p * ld + p], b = H[p * ld + p + 1], c = H[(p + 1) * ld + p], d = H[(p + 1) * ld + p + 1];
  R hm = 0.5 * (a - d);
  R disc = hm * hm + b * c;
  if (disc < 0.0 || c == 0.0) return;
  // eigenvalue closest to d: lambda = d + (hm +- se_sqrt(disc)) ... pick the one of larger magnitude shift
  R sq = se_sqrt(disc);
  R lam = 0.5 * (a + d) + (hm >= 0 ? sq : -sq);
  // eigenvector (lam - d, c) of the block; rotation taking it to e1
  R x = lam - d, y = c;
  R r = se_sqrt(x * x + y * y);
  if (r == 0.0) return;
  R cs = x / r, sn = y / r;
  // rows p, p+1: G^T H
  for (int col = p + t.lane; col < m; col += t.size) {
    R h1 = H[p * ld + col], h2 = H[(p + 1) * ld + col];
    H[p * ld + col] = cs * h1 + sn * h2;
    H[(p + 1) * ld + col] = -sn * h1 + cs * h2;
  }
  t.sync();
  for (int row = t.lane; row <= p + 1; row += t.size) {
    R h1 = H[row * ld + p], h2 = H[row * ld + p + 1];
    H[row * ld + p] = cs * h1 + sn * h2;
    H[row * ld + p + 1] = -sn * h1 + cs * h2;
  }
  for (int row = t.lane; row < m; row += t.size) {
    R q1 = Q[row * ldq + p], q2 = Q[row * ldq + p + 1];
    Q[row * ldq + p] = cs * q1 + sn * q2;
    Q[row * ldq + p + 1] = -sn * q1 + cs * q2;
  }
  t.sync();
  if (t.lane == 0) H[(p + 1) * ld + p] = 0.0;
  t.sync();
}

// Francis R-shift QR on an upper Hessenberg H, full Schur form, Q accumulated.
// A subdiagonal entry is neglected when it is below eps times its two diagonal
// neighbours or below eps times hnorm (the largest entry of the input), which keeps
// clusters of eigenvalues near zero from stalling the iteration; the result is
// backward stable relative to hnorm.  Returns 0 on success, -1 on no convergence.
// snap: 14 values of scratch shared by the team (may be null for a one-thread team).
// local_tol (>= the machine epsilon of R; 0 selects it): the neighbour-relative test may use a looser
// threshold when the caller needs the Schur form only to that relative accuracy; the test against
// hnorm always uses the machine epsilon.
template <class R>
SE_HD inline int schur(R* H, int ld, R* Q, int ldq, int m, double hnorm_, const Team& t, R* snap = nullptr,
                       double local_tol = 0.0) {
  R snap_local[14];
  if (!snap) snap = snap_local;
  const R eps = R(SeEps<R>::v), hnorm = R(hnorm_);
  const R leps = R(local_tol > SeEps<R>::v ? local_tol : SeEps<R>::v);
  int hi = m - 1, iter = 0, total = 0;
  while (hi >= 0) {
    int lo = hi;
    while (lo > 0) {
      R s = se_abs(H[(lo - 1) * ld + lo - 1]) + se_abs(H[lo * ld + lo]);
      const R sub = se_abs(H[lo * ld + lo - 1]);
      if (sub <= leps * s || sub <= eps * hnorm) break;
      --lo;
    }
    if (lo > 0) {
      t.sync();
      if (t.lane == 0) H[lo * ld + lo - 1] = 0.0;
      t.sync();
    }
    if (lo == hi) {
      --hi;
      iter = 0;
      continue;
    }
    if (lo == hi - 1) {
      split_2x2(H, ld, Q, ldq, m, lo, t);
      hi -= 2;
      iter = 0;
      continue;
    }
    ++iter;
    if (++total > 60 * m) return -1;
    // Shifts: the eigenvalues of the trailing 2x2 block (a real pair is replaced by its member
    // closer to the last diagonal entry, used twice), or an exceptional pair every 11th step.
    R s1r, s1i, s2r, s2i;
    {
      R a, b, c, d;
      if (iter % 11 == 10) {
        const R w = se_abs(H[hi * ld + hi - 1]) + se_abs(H[(hi - 1) * ld + hi - 2]);
        a = 0.75 * w + H[hi * ld + hi];
        b = -0.4375 * w;
        c = w;
        d = a;
      } else {
        a = H[(hi - 1) * ld + hi - 1];
        b = H[(hi - 1) * ld + hi];
        c = H[hi * ld + hi - 1];
        d = H[hi * ld + hi];
      }
      const R hm = 0.5 * (a - d);
      const R disc = hm * hm + b * c;
      const R mean = 0.5 * (a + d);
      if (disc >= 0.0) {
        const R sq = se_sqrt(disc);
        const R r1 = mean + sq, r2 = mean - sq;
        const R sh = (se_abs(r1 - d) <= se_abs(r2 - d)) ? r1 : r2;
        s1r = s2r = sh;
        s1i = s2i = 0.0;
      } else {
        s1r = s2r = mean;
        s1i = se_sqrt(-disc);
        s2i = -s1i;
      }
    }
    // first column of (H - s1)(H - s2), formed from differences to avoid cancellation
    R x, y, z;
    {
      const R h00 = H[lo * ld + lo], h01 = H[lo * ld + lo + 1], h10 = H[(lo + 1) * ld + lo];
      const R h11 = H[(lo + 1) * ld + lo + 1], h21 = H[(lo + 2) * ld + lo + 1];
      const R sc = se_abs(h00 - s2r) + se_abs(s2i) + se_abs(h10);
      const R g = (sc > 0.0) ? h10 / sc : 0.0;
      x = g * h01 + (h00 - s1r) * ((h00 - s2r) / (sc > 0.0 ? sc : 1.0)) - s1i * (s2i / (sc > 0.0 ? sc : 1.0));
      y = g * (h00 + h11 - s1r - s2r);
      z = g * h21;
    }
    // Bulge chase.  For k > lo the reflector is built from column k-1 (rows k..k+2), which it maps to
    // (alpha, 0, 0) exactly; that column is therefore not part of the left update but written
    // directly, after the barrier that separates every thread's read of (x, y, z) from the writes,
    // which keeps each step at two barriers.  The next step's reflector comes from column k after
    // this step's right update; one thread recomputes its three entries from a snapshot of rows
    // k+1..k+3 (columns k..k+2) taken in the left phase and forms the reflector while the others run
    // the right update, instead of every thread forming it after that update (the entries are the
    // values the right update writes).
    t.sync();  // the shift and deflation reads above precede the first update
    const bool early = SeEarlyReflector<R>::value;
    R u1, u2, beta, alpha;
    bool have = make_reflector(x, y, z, u1, u2, beta, alpha);
    for (int k = lo; k <= hi - 2; ++k) {
      const bool more = k + 1 <= hi - 2;  // a next step exists (then k + 3 <= hi)
      R nu1 = R(0.0), nu2 = R(0.0), nbeta = R(0.0), nalpha = R(0.0);
      bool nhave = false;
      if (have) {
        const int c0 = k > lo ? k : lo;
        const int r1 = (k + 3 <= hi) ? k + 3 : hi;
        // phase 1: rows k..k+2 from the left (columns c0..m-1) and the first qa rows of Q; phase 2:
        // columns k..k+2 from the right (rows 0..r1) and the remaining rows of Q (Q's update depends
        // on the reflector only, so it fills the threads that the H updates leave idle)
        const int ncol = m - c0;
        const int qa = (t.size > ncol) ? ((t.size - ncol < m) ? t.size - ncol : m) : 0;
        for (int idx = t.lane; idx < ncol + qa; idx += t.size) {
          R* a;
          int st;
          if (idx < ncol) {
            a = H + k * ld + c0 + idx;
            st = ld;
          } else {
            a = Q + (idx - ncol) * ldq + k;
            st = 1;
          }
          R d = a[0];
          se_mac(d, u1, a[st]);
          se_mac(d, u2, a[2 * st]);
          d = se_fin(d) * beta;
          a[0] -= d;
          a[st] -= d * u1;
          a[2 * st] -= d * u2;
          if (early && more && idx < 3) {  // column c0 + idx = k + idx
            snap[idx] = a[st];
            snap[3 + idx] = a[2 * st];
            snap[6 + idx] = H[(k + 3) * ld + k + idx];
          }
        }
        t.sync();
        if (k > lo && t.lane == 0) {
          H[k * ld + k - 1] = alpha;
          H[(k + 1) * ld + k - 1] = 0.0;
          H[(k + 2) * ld + k - 1] = 0.0;
        }
        if (early && more && t.lane == t.size - 1) {  // the last thread, usually idle in the right update
          R v[3];
          for (int rr = 0; rr < 3; ++rr) {
            const R a0 = snap[3 * rr], a1 = snap[3 * rr + 1], a2 = snap[3 * rr + 2];
            R d = a0;
            se_mac(d, u1, a1);
            se_mac(d, u2, a2);
            d = se_fin(d) * beta;
            v[rr] = a0 - d;
          }
          const bool ok = make_reflector(v[0], v[1], v[2], nu1, nu2, nbeta, nalpha);
          snap[9] = nu1;
          snap[10] = nu2;
          snap[11] = nbeta;
          snap[12] = nalpha;
          snap[13] = ok ? R(1.0) : R(0.0);
        }
        for (int idx = t.lane; idx < (r1 + 1) + (m - qa); idx += t.size) {
          R* a = (idx <= r1) ? H + idx * ld + k : Q + (qa + idx - (r1 + 1)) * ldq + k;
          R d = a[0];
          se_mac(d, u1, a[1]);
          se_mac(d, u2, a[2]);
          d = se_fin(d) * beta;
          a[0] -= d;
          a[1] -= d * u1;
          a[2] -= d * u2;
        }
        t.sync();
        if (more && early) {
          nu1 = snap[9];
          nu2 = snap[10];
          nbeta = snap[11];
          nalpha = snap[12];
          nhave = snap[13] != R(0.0);
        } else if (more) {
          nhave = make_reflector(H[(k + 1) * ld + k], H[(k + 2) * ld + k], H[(k + 3) * ld + k], nu1, nu2, nbeta,
                                 nalpha);
        }
      } else if (more) {
        nhave = make_reflector(H[(k + 1) * ld + k], H[(k + 2) * ld + k], H[(k + 3) * ld + k], nu1, nu2, nbeta,
                               nalpha);
      }
      u1 = nu1;
      u2 = nu2;
      beta = nbeta;
      alpha = nalpha;
      have = nhave;
    }
    x = H[(hi - 1) * ld + hi - 2];
    y = H[hi * ld + hi - 2];
    // final 2-element reflector on rows hi-1, hi
    {
      R u1, u2, beta, alpha;
      if (make_reflector<R>(x, y, R(0.0), u1, u2, beta, alpha)) {
        t.sync();
        apply_reflector<R>(H, ld, Q, ldq, m, hi - 1, 2, u1, R(0.0), beta, hi - 2, hi, t);
        if (t.lane == 0) H[hi * ld + hi - 2] = 0.0;
        t.sync();
      }
    }
  }
  return 0;
}

// Eigenvalues of the quasi-triangular S: wr[j], wi[j] (a complex pair occupies j, j+1 with wi[j] > 0).
template <class R>
SE_HD inline void schur_eigenvalues(const R* S, int ld, int m, double* wr, double* wi) {
  int j = 0;
  while (j < m) {
    if (j + 1 < m && S[(j + 1) * ld + j] != 0.0) {
      R a = S[j * ld + j], b = S[j * ld + j + 1], c = S[(j + 1) * ld + j], d = S[(j + 1) * ld + j + 1];
      R hm = 0.5 * (a - d);
      R disc = hm * hm + b * c;
      R re = 0.5 * (a + d);
      R im = se_sqrt(se_abs(disc));
      if (disc >= 0.0) {  // not split (should not happen after split_2x2); report real values
        wr[j] = se_dbl(re + im);
        wr[j + 1] = se_dbl(re - im);
        wi[j] = wi[j + 1] = 0.0;
      } else {
        wr[j] = wr[j + 1] = se_dbl(re);
        wi[j] = se_dbl(im);
        wi[j + 1] = -se_dbl(im);
      }
      j += 2;
    } else {
      wr[j] = se_dbl(S[j * ld + j]);
      wi[j] = 0.0;
      j += 1;
    }
  }
}

// Eigenvector of the quasi-triangular S for the eigenvalue at position p (real: x; complex
// pair starting at p: x + i y).  x, y have m entries; entries above p are filled, below zero.
template <class R>
SE_HD inline void schur_vector(const R* S, int ld, int m, int p, double lr_, double li_, R* x, R* y,
                               double snorm) {
  const R small = R(1e-300 + SeEps<R>::v * snorm);
  const R lr = R(lr_), li = R(li_);
  for (int q = 0; q < m; ++q) {
    x[q] = 0.0;
    y[q] = 0.0;
  }
  int top;
  if (li == 0.0) {
    x[p] = 1.0;
    top = p - 1;
  } else {
    // block rows p, p+1: (a - lambda) x_p + b x_{p+1} = 0 -> x_p = b, x_{p+1} = lambda - a
    R a = S[p * ld + p], b = S[p * ld + p + 1];
    x[p] = b;
    y[p] = 0.0;
    x[p + 1] = lr - a;
    y[p + 1] = li;
    top = p - 1;
  }
  const int last = (li == 0.0) ? p : p + 1;
  R mx = 0.0;
  for (int c = top + 1; c <= last; ++c) {
    const R v = se_abs(x[c]) + se_abs(y[c]);
    if (v > mx) mx = v;
  }
  int q = top;
  while (q >= 0) {
    if (q > 0 && S[q * ld + q - 1] != 0.0) {
      // 2x2 block rows q-1, q: solve (S_blk - lambda I) [u; w] = -rhs
      R r1r = 0, r1i = 0, r2r = 0, r2i = 0;
      for (int c = q + 1; c <= last; ++c) {
        se_mac(r1r, S[(q - 1) * ld + c], x[c]);
        se_mac(r1i, S[(q - 1) * ld + c], y[c]);
        se_mac(r2r, S[q * ld + c], x[c]);
        se_mac(r2i, S[q * ld + c], y[c]);
      }
      r1r = se_fin(r1r);
      r1i = se_fin(r1i);
      r2r = se_fin(r2r);
      r2i = se_fin(r2i);
      R a11r = S[(q - 1) * ld + q - 1] - lr, a11i = -li;
      R a12 = S[(q - 1) * ld + q], a21 = S[q * ld + q - 1];
      R a22r = S[q * ld + q] - lr, a22i = -li;
      // det = a11*a22 - a12*a21 (complex)
      R dr = a11r * a22r - a11i * a22i - a12 * a21;
      R di = a11r * a22i + a11i * a22r;
      R dn = dr * dr + di * di;
      if (dn < small * small) {
        dr = small;
        di = 0.0;
        dn = small * small;
      }
      // [u; w] = -inv(A) r,  inv(A) = [a22 -a12; -a21 a11] / det
      R ur = -(a22r * r1r - a22i * r1i - a12 * r2r);
      R ui = -(a22r * r1i + a22i * r1r - a12 * r2i);
      R wr_ = -(-a21 * r1r + a11r * r2r - a11i * r2i);
      R wi_ = -(-a21 * r1i + a11r * r2i + a11i * r2r);
      x[q - 1] = (ur * dr + ui * di) / dn;
      y[q - 1] = (ui * dr - ur * di) / dn;
      x[q] = (wr_ * dr + wi_ * di) / dn;
      y[q] = (wi_ * dr - wr_ * di) / dn;
      q -= 2;
    } else {
      R rr = 0, ri = 0;
      for (int c = q + 1; c <= last; ++c) {
        se_mac(rr, S[q * ld + c], x[c]);
        se_mac(ri, S[q * ld + c], y[c]);
      }
      rr = se_fin(rr);
      ri = se_fin(ri);
      R dr = S[q * ld + q] - lr, di = -li;
      R dn = dr * dr + di * di;
      if (dn < small * small) {
        dr = small;
        di = 0.0;
        dn = small * small;
      }
      x[q] = -(rr * dr + ri * di) / dn;
      y[q] = -(ri * dr - rr * di) / dn;
      q -= 1;
    }
    // rescale to avoid overflow: mx is the largest |x_c| + |y_c| over the entries computed so far
    for (int c = q + 1; c <= q + 2 && c <= last; ++c) {
      const R v = se_abs(x[c]) + se_abs(y[c]);
      if (v > mx) mx = v;
    }
    if (mx > R(SeEps<R>::big)) {
      const R inv = R(1.0) / mx;
      for (int c = 0; c <= last; ++c) {
        x[c] *= inv;
        y[c] *= inv;
      }
      mx = R(1.0);
    }
  }
}

// Order of eigenvalues by decreasing modulus; within a pair the +imag member first.
// perm: m ints; mod: m doubles of scratch.  Selection sort (m is small).
SE_HD inline void order_by_modulus(const double* wr, const double* wi, int m, int* perm, double* mod) {
  for (int j = 0; j < m; ++j) {
    perm[j] = j;
    mod[j] = hypot(wr[j], wi[j]);
  }
  for (int a = 0; a < m; ++a) {
    int best = a;
    double bm = mod[perm[a]];
    for (int b = a + 1; b < m; ++b) {
      const double mb = mod[perm[b]];
      if (mb > bm * (1 + 1e-14) || (fabs(mb - bm) <= 1e-14 * bm && wi[perm[b]] > wi[perm[best]])) {
        best = b;
        bm = mb;
      }
    }
    const int tmp = perm[a];
    perm[a] = perm[best];
    perm[best] = tmp;
  }
}

}  // namespace se
}  // namespace a2ls
