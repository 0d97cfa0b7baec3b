// Prints host-built operator chains as dense matrices for the CPU tests:
// argv: kind L vmin dv nu u vth.  kind: coll | coll_reduced | d2
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "mpo_build.hpp"

using namespace vp;

int main(int argc, char** argv) {
  if (argc != 8) return 2;
  const int L = std::atoi(argv[2]);
  const double vmin = std::atof(argv[3]), dv = std::atof(argv[4]), nu = std::atof(argv[5]), u = std::atof(argv[6]),
               vth = std::atof(argv[7]);
  Chain c;
  if (!std::strcmp(argv[1], "d2")) c = second_zero_gradient_chain(L, dv);
  else c = collision_chain(L, vmin, dv, nu, u, vth);
  if (!std::strcmp(argv[1], "coll_reduced")) c = reduce_chain(c, 1e-13);
  printf("bonds");
  for (int w : c.w) printf(" %d", w);
  printf("\n");
  const int N = 1 << L;
  for (int o = 0; o < N; ++o) {
    for (int i = 0; i < N; ++i) {
      std::vector<double> v(1, 1.0);
      for (int k = 0; k < L; ++k) {
        const int ob = (o >> (L - 1 - k)) & 1, ib = (i >> (L - 1 - k)) & 1;
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
