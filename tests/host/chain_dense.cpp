// Prints host-built operator chains as dense matrices for the CPU tests:
// argv: kind L vmin dv nu u vth [nx dx mapping].  kind: coll | coll_reduced |
// d2 | static (the upwind operator plus the placed collision chain, reduced,
// as a collisional species' sim builds it; mapping 0 S1, 1 IF, 2 S2, 3 S3).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "mpo_build.hpp"

using namespace vp;

int main(int argc, char** argv) {
  if (argc != 8 && argc != 11) return 2;
  const int L = std::atoi(argv[2]);
  const double vmin = std::atof(argv[3]), dv = std::atof(argv[4]), nu = std::atof(argv[5]), u = std::atof(argv[6]),
               vth = std::atof(argv[7]);
  Chain c;
  int nsites = L;
  if (!std::strcmp(argv[1], "d2")) {
    c = second_zero_gradient_chain(L, dv);
  } else if (!std::strcmp(argv[1], "static")) {
    if (argc != 11) return 2;
    const int nx = std::atoi(argv[8]), mapping = std::atoi(argv[10]);
    const double dx = std::atof(argv[9]);
    std::vector<int> dims;
    if (mapping == 1) {
      for (int b = 0; b < (nx > L ? nx : L); ++b) {
        if (b < nx) dims.push_back(0);
        if (b < L) dims.push_back(1);
      }
    } else {
      for (int b = 0; b < nx; ++b) dims.push_back(0);
      for (int b = 0; b < L; ++b) dims.push_back(1);
    }
    const bool xd = mapping == 2, vd = mapping == 3;
    Chain cv = collision_chain(L, vmin, dv, nu, u, vth);
    if (vd) cv = reverse_chain(cv);
    c = reduce_chain(chain_sum(upwind_operator(nx, L, dims, dx, vmin, dv, xd, vd), place2(identity_chain(nx), cv, dims)),
                     1e-13);
    nsites = nx + L;
  } else {
    c = collision_chain(L, vmin, dv, nu, u, vth);
  }
  if (!std::strcmp(argv[1], "coll_reduced")) c = reduce_chain(c, 1e-13);
  printf("bonds");
  for (int w : c.w) printf(" %d", w);
  printf("\n");
  const int N = 1 << nsites;
  for (int o = 0; o < N; ++o) {
    for (int i = 0; i < N; ++i) {
      std::vector<double> v(1, 1.0);
      for (int k = 0; k < nsites; ++k) {
        const int ob = (o >> (nsites - 1 - k)) & 1, ib = (i >> (nsites - 1 - k)) & 1;
        std::vector<double> nv(c.w[k + 1], 0.0);
        for (int l = 0; l < c.w[k]; ++l)
          for (int r = 0; r < c.w[k + 1]; ++r) nv[r] += v[l] * c.core[k][((size_t)l * 4 + ob * 2 + ib) * c.w[k + 1] + r];
        v = nv;
      }
      printf("%.17g ", v[0]);
    }
    printf("\n");
  }
  return 0;
}
