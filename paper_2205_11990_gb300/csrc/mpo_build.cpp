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
