// Host construction of the finite-difference MPOs of the Vlasov operator.
#pragma once

#include <vector>

namespace vp {

// An MPO chain over L bits (most significant first): cores (wl, 2_out, 2_in, wr)
// row-major, bonds w[0..L] with w[0] = w[L] = 1 unless stated.
struct Chain {
  std::vector<int> w;
  std::vector<std::vector<double>> core;
  double& at(int k, int l, int o, int i, int r) { return core[k][((size_t)l * 4 + o * 2 + i) * w[k + 1] + r]; }
  void alloc(const std::vector<int>& bonds) {
    w = bonds;
    core.assign(w.size() - 1, {});
    for (size_t k = 0; k + 1 < w.size(); ++k) core[k].assign((size_t)w[k] * 4 * w[k + 1], 0.0);
  }
};

// Shift stencil sum_s c[s+2] * (f_{n+s}), s = -2..2, on L bits, as a carry
// automaton with three channels (carry 0, +1, -1); periodic or not.  The last
// core maps onto `nout` right channels with one coefficient set per channel
// (coeffs[t][s+2]), so several stencils can share the carry propagation.
Chain stencil_chain(int L, const std::vector<std::vector<double>>& coeffs, bool periodic);
// Centred first derivative with zero-gradient ends (ghost node equal to the
// node inside the boundary): derivative zero on the first and last node.
Chain zero_gradient_chain(int L, double dv);
// Three-point second derivative with the same mirrored ghosts.
Chain second_zero_gradient_chain(int L, double dv);
// The operator a b (b applied first); bonds multiply.
Chain chain_product(const Chain& a, const Chain& b);
// Dougherty collision operator on the v bits (Methods, "Collision Operator"):
// nu [D_c diag(v - u) + vth^2 D_vv], both derivatives zero-gradient.
Chain collision_chain(int L, double vmin, double dv, double nu, double u, double vth);
// The same operator with every bond reduced to its numerical rank: an SVD
// sweep left to right, then right to left, dropping singular values at or
// below rel times the largest of their bond (host, small cores only).
Chain reduce_chain(const Chain& c, double rel);
// diag(v * h(v_msb)) on L bits, v_j = vmin + j dv, h selects v > 0 (upper
// half) when positive, else v < 0; as an affine chain of bond 2.  If
// left_channels == 2 the first core takes a 2-channel left bond with
// channel 0 = backward/positive and 1 = forward/negative (upwind split).
Chain velocity_chain(int L, double vmin, double dv, int which);

// Upwind advection -v+ D_b^x - v- D_f^x on the full site chain.
// sitemap[k] = 0 for an x bit, 1 for a v bit (bits in order).
Chain upwind_operator(int nx, int nv, const std::vector<int>& sitedim, double dx, double vmin, double dv,
                      bool xdesc = false, bool vdesc = false);

// Generic placement of per-dimension chains on the site order (tensor
// product; bonds multiply, dimension 0 index major).
Chain place2(const Chain& X, const Chain& V, const std::vector<int>& sitedim);
Chain chain_sum(const Chain& a, const Chain& b);
Chain identity_chain(int L);
// The same operator with its sites in the opposite order (core k <- core L-1-k,
// bonds exchanged): for a dimension whose bits appear fine to coarse.
Chain reverse_chain(const Chain& a);
Chain scaled(const Chain& a, double s);

}  // namespace vp
