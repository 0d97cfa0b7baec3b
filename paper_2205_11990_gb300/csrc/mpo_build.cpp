// Host construction of the finite-difference MPOs (SI "Derivatives", "Upwind
// time evolution").  The cores are not transcribed from the printed chains:
// each stencil is built as a carry automaton.  With bits most significant
// first, a shift in = out + s is realised bit by bit from the least
// significant end: at a bit with outgoing carry o_r (from the less
// significant bits) and incoming carry o_l (to the more significant ones),
// out bit n and in bit m must satisfy n + o_r - m = 2 o_l.  For |s| <= 2 the
// carries stay in {-1, 0, +1}, hence bond 3; the most significant bit drops
// its carry (periodic) or requires it to vanish (non-periodic).
#include "mpo_build.hpp"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace vp {

static const int kOff[3] = {0, 1, -1};  // carry of channel 0, 1, 2

static bool msb_ok(int n, int o_r, int m, bool periodic) {
  const int d = n + o_r - m;
  return periodic ? (d % 2 == 0) : (d == 0);
}

Chain stencil_chain(int L, const std::vector<std::vector<double>>& coeffs, bool periodic) {
  const int nout = (int)coeffs.size();
  std::vector<int> w(L + 1, 3);
  w[0] = 1;
  w[L] = nout;
  Chain c;
  c.alloc(w);
  for (int k = 0; k < L; ++k) {
    const bool msb = (k == 0), lsb = (k == L - 1);
    for (int l = 0; l < w[k]; ++l)
      for (int n = 0; n < 2; ++n)
        for (int m = 0; m < 2; ++m) {
          if (!lsb) {
            for (int r = 0; r < 3; ++r) {
              const bool ok = msb ? msb_ok(n, kOff[r], m, periodic) : (n + kOff[r] - m == 2 * kOff[l]);
              if (ok) c.at(k, l, n, m, r) = 1.0;
            }
          } else {
            for (int t = 0; t < nout; ++t) {
              double v = 0.0;
              for (int s = -2; s <= 2; ++s) {
                const double cs = coeffs[t][s + 2];
                if (cs == 0.0) continue;
                const bool ok = msb ? msb_ok(n, s, m, periodic) : (n + s - m == 2 * kOff[l]);
                if (ok) v += cs;
              }
              c.at(k, l, n, m, t) = v;
            }
          }
        }
  }
  return c;
}

// Non-periodic stencil sum_s c_s f_{n+s} plus ghost corrections on the end
// rows: row 0 gains first * f_1, row N-1 gains last * f_{N-2} (the mirrored
// ghosts f_{-1} = f_1 and f_N = f_{N-2} folded back onto the grid).
static Chain ghost_chain(int L, const std::vector<double>& co, double first, double last) {
  Chain base = stencil_chain(L, {co}, false);
  if (L == 1) {
    base.at(0, 0, 0, 1, 0) += first;
    base.at(0, 0, 1, 0, 0) += last;
    return base;
  }
  std::vector<int> w(L + 1, 5);
  w[0] = 1;
  w[L] = 1;
  Chain c;
  c.alloc(w);
  for (int k = 0; k < L; ++k) {
    const bool msb = (k == 0), lsb = (k == L - 1);
    // carry channels copied from the plain non-periodic stencil
    for (int l = 0; l < base.w[k]; ++l)
      for (int n = 0; n < 2; ++n)
        for (int m = 0; m < 2; ++m)
          for (int r = 0; r < base.w[k + 1]; ++r) c.at(k, l, n, m, r) = base.at(k, l, n, m, r);
    // channel 3: all bits 0 (row 0), channel 4: all bits 1 (row N-1)
    if (msb) {
      c.at(k, 0, 0, 0, 3) = 1.0;
      c.at(k, 0, 1, 1, 4) = 1.0;
    } else if (!lsb) {
      c.at(k, 3, 0, 0, 3) = 1.0;
      c.at(k, 4, 1, 1, 4) = 1.0;
    } else {
      c.at(k, 3, 0, 1, 0) = first;
      c.at(k, 4, 1, 0, 0) = last;
    }
  }
  return c;
}

Chain zero_gradient_chain(int L, double dv) {
  const double c1 = 0.5 / dv;
  // row 0 loses +c1 f_1 (ghost f_{-1} = f_1), row N-1 loses -c1 f_{N-2}
  return ghost_chain(L, {0.0, -c1, 0.0, c1, 0.0}, -c1, c1);
}

Chain second_zero_gradient_chain(int L, double dv) {
  const double s = 1.0 / (dv * dv);
  // the ghosts add s f_1 to row 0 and s f_{N-2} to row N-1
  return ghost_chain(L, {0.0, s, -2.0 * s, s, 0.0}, s, s);
}

Chain chain_product(const Chain& a, const Chain& b) {
  const int L = (int)a.core.size();
  std::vector<int> w(L + 1);
  for (int k = 0; k <= L; ++k) w[k] = a.w[k] * b.w[k];
  Chain c;
  c.alloc(w);
  for (int k = 0; k < L; ++k) {
    const int al = a.w[k], ar = a.w[k + 1], bl = b.w[k], br = b.w[k + 1];
    for (int la = 0; la < al; ++la)
      for (int ra = 0; ra < ar; ++ra)
        for (int o = 0; o < 2; ++o)
          for (int j = 0; j < 2; ++j) {
            const double x = a.core[k][((size_t)la * 4 + o * 2 + j) * ar + ra];
            if (x == 0.0) continue;
            for (int lb = 0; lb < bl; ++lb)
              for (int rb = 0; rb < br; ++rb)
                for (int i = 0; i < 2; ++i) {
                  const double y = b.core[k][((size_t)lb * 4 + j * 2 + i) * br + rb];
                  if (y != 0.0) c.at(k, la * bl + lb, o, i, ra * br + rb) += x * y;
                }
          }
  }
  return c;
}

// Thin SVD of a small row-major m x n matrix by one-sided (Hestenes)
// Jacobi rotations on the columns of A (m >= n) or of A^T (m < n):
// A = U diag(s) Vt, s descending, U m x k, Vt k x n, k = min(m, n).
static void small_svd(int m, int n, const std::vector<double>& A, std::vector<double>& U, std::vector<double>& s,
                      std::vector<double>& Vt) {
  const bool tr = m < n;
  const int R = tr ? n : m, C = tr ? m : n;  // work on W (R x C), R >= C
  std::vector<double> W((size_t)R * C), V((size_t)C * C, 0.0);
  for (int i = 0; i < R; ++i)
    for (int j = 0; j < C; ++j) W[(size_t)i * C + j] = tr ? A[(size_t)j * n + i] : A[(size_t)i * n + j];
  for (int j = 0; j < C; ++j) V[(size_t)j * C + j] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < C - 1; ++p)
      for (int q = p + 1; q < C; ++q) {
        double a = 0, b = 0, g = 0;
        for (int i = 0; i < R; ++i) {
          const double x = W[(size_t)i * C + p], y = W[(size_t)i * C + q];
          a += x * x;
          b += y * y;
          g += x * y;
        }
        if (g == 0.0 || std::fabs(g) <= 1e-15 * std::sqrt(a * b)) continue;
        off = std::max(off, std::fabs(g) / std::sqrt(a * b));
        const double zeta = (b - a) / (2.0 * g);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        for (int i = 0; i < R; ++i) {
          const double x = W[(size_t)i * C + p], y = W[(size_t)i * C + q];
          W[(size_t)i * C + p] = c * x - sn * y;
          W[(size_t)i * C + q] = sn * x + c * y;
        }
        for (int i = 0; i < C; ++i) {
          const double x = V[(size_t)i * C + p], y = V[(size_t)i * C + q];
          V[(size_t)i * C + p] = c * x - sn * y;
          V[(size_t)i * C + q] = sn * x + c * y;
        }
      }
    if (off <= 1e-15) break;
  }
  std::vector<int> ord(C);
  std::vector<double> nrm(C);
  for (int j = 0; j < C; ++j) {
    double a = 0;
    for (int i = 0; i < R; ++i) a += W[(size_t)i * C + j] * W[(size_t)i * C + j];
    nrm[j] = std::sqrt(a);
    ord[j] = j;
  }
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return nrm[x] > nrm[y]; });
  // W = Ul S with Ul = W / s column-wise; A = W V^T (or A^T = W V^T)
  std::vector<double> Ul((size_t)R * C, 0.0);
  s.assign(C, 0.0);
  for (int jj = 0; jj < C; ++jj) {
    const int j = ord[jj];
    s[jj] = nrm[j];
    if (nrm[j] > 0)
      for (int i = 0; i < R; ++i) Ul[(size_t)i * C + jj] = W[(size_t)i * C + j] / nrm[j];
  }
  if (!tr) {  // A = Ul S V^T
    U = Ul;
    Vt.assign((size_t)C * n, 0.0);
    for (int jj = 0; jj < C; ++jj)
      for (int i = 0; i < n; ++i) Vt[(size_t)jj * n + i] = V[(size_t)i * C + ord[jj]];
  } else {  // A^T = Ul S V^T  =>  A = V S Ul^T
    U.assign((size_t)m * C, 0.0);
    for (int i = 0; i < m; ++i)
      for (int jj = 0; jj < C; ++jj) U[(size_t)i * C + jj] = V[(size_t)i * C + ord[jj]];
    Vt.assign((size_t)C * n, 0.0);
    for (int jj = 0; jj < C; ++jj)
      for (int i = 0; i < n; ++i) Vt[(size_t)jj * n + i] = Ul[(size_t)i * C + jj];
  }
}

Chain reduce_chain(const Chain& in, double rel) {
  Chain c = in;
  const int L = (int)c.core.size();
  auto keep = [&](const std::vector<double>& s) {
    int r = 0;
    while (r < (int)s.size() && s[r] > rel * s[0]) ++r;
    return std::max(r, 1);
  };
  std::vector<double> U, s, Vt;
  // left to right: core k = U (S Vt), S Vt absorbed into core k+1
  for (int k = 0; k + 1 < L; ++k) {
    const int wl = c.w[k], wr = c.w[k + 1], m = wl * 4;
    small_svd(m, wr, c.core[k], U, s, Vt);
    const int kk = std::min(m, wr), r = keep(s);
    std::vector<double> ck((size_t)m * r);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < r; ++j) ck[(size_t)i * r + j] = U[(size_t)i * kk + j];
    const int wn = c.w[k + 2];
    std::vector<double> nx((size_t)r * 4 * wn, 0.0);
    for (int j = 0; j < r; ++j)
      for (int t = 0; t < wr; ++t) {
        const double f = s[j] * Vt[(size_t)j * wr + t];
        if (f == 0.0) continue;
        for (int e = 0; e < 4 * wn; ++e) nx[(size_t)j * 4 * wn + e] += f * c.core[k + 1][(size_t)t * 4 * wn + e];
      }
    c.core[k] = ck;
    c.core[k + 1] = nx;
    c.w[k + 1] = r;
  }
  // right to left: core k = (U S) Vt, U S absorbed into core k-1
  for (int k = L - 1; k > 0; --k) {
    const int wl = c.w[k], wr = c.w[k + 1], n = 4 * wr;
    small_svd(wl, n, c.core[k], U, s, Vt);
    const int kk = std::min(wl, n), r = keep(s);
    std::vector<double> ck((size_t)r * n);
    for (int j = 0; j < r; ++j)
      for (int e = 0; e < n; ++e) ck[(size_t)j * n + e] = Vt[(size_t)j * n + e];
    const int wp = c.w[k - 1];
    std::vector<double> pv((size_t)wp * 4 * r, 0.0);
    for (int a = 0; a < wp * 4; ++a)
      for (int t = 0; t < wl; ++t) {
        const double x = c.core[k - 1][(size_t)a * wl + t];
        if (x == 0.0) continue;
        for (int j = 0; j < r; ++j) pv[(size_t)a * r + j] += x * U[(size_t)t * kk + j] * s[j];
      }
    c.core[k] = ck;
    c.core[k - 1] = pv;
    c.w[k] = r;
  }
  return c;
}

Chain collision_chain(int L, double vmin, double dv, double nu, double u, double vth) {
  Chain drag = chain_product(zero_gradient_chain(L, dv), velocity_chain(L, vmin - u, dv, 0));
  Chain c = chain_sum(drag, scaled(second_zero_gradient_chain(L, dv), vth * vth));
  return scaled(c, nu);
}

static double hsel(int which, int bit) {
  if (which > 0) return bit == 1 ? 1.0 : 0.0;
  if (which < 0) return bit == 0 ? 1.0 : 0.0;
  return 1.0;
}

Chain velocity_chain(int L, double vmin, double dv, int which) {
  Chain c;
  if (L == 1) {
    c.alloc({1, 1});
    for (int n = 0; n < 2; ++n) c.at(0, 0, n, n, 0) = hsel(which, n) * (vmin + dv * n);
    return c;
  }
  std::vector<int> w(L + 1, 2);
  w[0] = 1;
  w[L] = 1;
  c.alloc(w);
  for (int n = 0; n < 2; ++n) {
    const double h = hsel(which, n);
    c.at(0, 0, n, n, 0) = h * (vmin + dv * n * std::ldexp(1.0, L - 1));
    c.at(0, 0, n, n, 1) = h;
    for (int k = 1; k < L - 1; ++k) {
      c.at(k, 0, n, n, 0) = 1.0;
      c.at(k, 1, n, n, 0) = dv * n * std::ldexp(1.0, L - 1 - k);
      c.at(k, 1, n, n, 1) = 1.0;
    }
    c.at(L - 1, 0, n, n, 0) = 1.0;
    c.at(L - 1, 1, n, n, 0) = dv * n;
  }
  return c;
}

Chain identity_chain(int L) {
  Chain c;
  c.alloc(std::vector<int>(L + 1, 1));
  for (int k = 0; k < L; ++k) {
    c.at(k, 0, 0, 0, 0) = 1.0;
    c.at(k, 0, 1, 1, 0) = 1.0;
  }
  return c;
}

Chain reverse_chain(const Chain& a) {
  const int L = (int)a.core.size();
  std::vector<int> w(L + 1);
  for (int k = 0; k <= L; ++k) w[k] = a.w[L - k];
  Chain c;
  c.alloc(w);
  for (int k = 0; k < L; ++k) {
    const int src = L - 1 - k;
    const int al = a.w[src], ar = a.w[src + 1];
    for (int l = 0; l < al; ++l)
      for (int r = 0; r < ar; ++r)
        for (int oi = 0; oi < 4; ++oi) c.core[k][((size_t)r * 4 + oi) * al + l] = a.core[src][((size_t)l * 4 + oi) * ar + r];
  }
  return c;
}

Chain scaled(const Chain& a, double s) {
  Chain c = a;
  for (double& x : c.core[0]) x *= s;
  return c;
}

Chain place2(const Chain& X, const Chain& V, const std::vector<int>& sitedim) {
  const int n = (int)sitedim.size();
  std::vector<int> w(n + 1);
  int px = 0, pv = 0;
  w[0] = X.w[0] * V.w[0];
  for (int k = 0; k < n; ++k) {
    if (sitedim[k] == 0) ++px; else ++pv;
    w[k + 1] = X.w[px] * V.w[pv];
  }
  Chain c;
  c.alloc(w);
  px = pv = 0;
  for (int k = 0; k < n; ++k) {
    if (sitedim[k] == 0) {
      const int dw = V.w[pv];
      const int al = X.w[px], ar = X.w[px + 1];
      for (int a = 0; a < al; ++a)
        for (int b = 0; b < ar; ++b)
          for (int o = 0; o < 2; ++o)
            for (int i = 0; i < 2; ++i) {
              const double v = X.core[px][((size_t)a * 4 + o * 2 + i) * ar + b];
              if (v == 0.0) continue;
              for (int d = 0; d < dw; ++d) c.at(k, a * dw + d, o, i, b * dw + d) = v;
            }
      ++px;
    } else {
      const int ew = X.w[px];
      const int al = V.w[pv], ar = V.w[pv + 1];
      for (int a = 0; a < al; ++a)
        for (int b = 0; b < ar; ++b)
          for (int o = 0; o < 2; ++o)
            for (int i = 0; i < 2; ++i) {
              const double v = V.core[pv][((size_t)a * 4 + o * 2 + i) * ar + b];
              if (v == 0.0) continue;
              for (int e = 0; e < ew; ++e) c.at(k, e * al + a, o, i, e * ar + b) = v;
            }
      ++pv;
    }
  }
  return c;
}

Chain chain_sum(const Chain& a, const Chain& b) {
  const int n = (int)a.core.size();
  std::vector<int> w(n + 1);
  w[0] = 1;
  w[n] = 1;
  for (int k = 1; k < n; ++k) w[k] = a.w[k] + b.w[k];
  Chain c;
  c.alloc(w);
  for (int k = 0; k < n; ++k) {
    const int ol = (k == 0) ? 0 : a.w[k];          // left offset of b
    const int orr = (k == n - 1) ? 0 : a.w[k + 1];  // right offset of b
    for (int src = 0; src < 2; ++src) {
      const Chain& s = src ? b : a;
      const int offl = src ? ol : 0, offr = src ? orr : 0;
      for (int l = 0; l < s.w[k]; ++l)
        for (int r = 0; r < s.w[k + 1]; ++r)
          for (int oi = 0; oi < 4; ++oi)
            c.core[k][((size_t)(l + offl) * 4 + oi) * w[k + 1] + r + offr] +=
                s.core[k][((size_t)l * 4 + oi) * s.w[k + 1] + r];
    }
  }
  return c;
}

Chain upwind_operator(int nx, int nv, const std::vector<int>& sitedim, double dx, double vmin, double dv,
                      bool xdesc, bool vdesc) {
  // v > 0: backward stencil (3 f_n - 4 f_{n-1} + f_{n-2}) / (2 dx);
  // v < 0: forward stencil (-3 f_n + 4 f_{n+1} - f_{n+2}) / (2 dx)
  const std::vector<double> cb = {0.5 / dx, -2.0 / dx, 1.5 / dx, 0.0, 0.0};
  const std::vector<double> cf = {0.0, 0.0, -1.5 / dx, 2.0 / dx, -0.5 / dx};
  bool seq = !xdesc && !vdesc;
  for (int k = 0; k < (int)sitedim.size(); ++k) seq = seq && (sitedim[k] == (k < nx ? 0 : 1));
  if (!seq) {
    auto ox = [&](Chain c) { return xdesc ? reverse_chain(c) : c; };
    auto ov = [&](Chain c) { return vdesc ? reverse_chain(c) : c; };
    Chain b = place2(ox(stencil_chain(nx, {cb}, true)), ov(scaled(velocity_chain(nv, vmin, dv, +1), -1.0)), sitedim);
    Chain f = place2(ox(stencil_chain(nx, {cf}, true)), ov(scaled(velocity_chain(nv, vmin, dv, -1), -1.0)), sitedim);
    return chain_sum(b, f);
  }
  // Sequential sites: the two stencils share the x carry channels and end on
  // a two-channel junction (0 = backward, 1 = forward); the velocity factors
  // v H(v) and v (1 - H(v)) share the affine channels after the first v bit.
  Chain X = stencil_chain(nx, {cb, cf}, true);
  Chain Vp = velocity_chain(nv, vmin, dv, +1), Vm = velocity_chain(nv, vmin, dv, -1);
  std::vector<int> w(nx + nv + 1);
  for (int k = 0; k <= nx; ++k) w[k] = X.w[k];
  for (int k = 1; k <= nv; ++k) w[nx + k] = Vp.w[k];
  Chain c;
  c.alloc(w);
  for (int k = 0; k < nx; ++k) c.core[k] = X.core[k];
  for (int k = 0; k < nv; ++k) {
    if (k == 0) {
      for (int t = 0; t < 2; ++t) {
        const Chain& V = t == 0 ? Vp : Vm;
        for (int n = 0; n < 2; ++n)
          for (int r = 0; r < w[nx + 1]; ++r)
            c.at(nx, t, n, n, r) = -V.core[0][((size_t)0 * 4 + n * 2 + n) * V.w[1] + r];
      }
    } else {
      c.core[nx + k] = Vp.core[k];
    }
  }
  return c;
}

}  // namespace vp
