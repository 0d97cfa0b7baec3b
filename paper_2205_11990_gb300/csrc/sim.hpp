// Internal: the simulation object of vp_sim_* and the MPS helpers that the
// stepping code of api.cu and the lockstep group of group.cu share.
#pragma once

#include <vector>

#include "common.cuh"
#include "mpo_build.hpp"

namespace vp {

// Flop counters of the factorisations (algorithmic counts).
struct Flops {
  double qr = 0, formq = 0, gemm = 0, jacobi = 0;
};

size_t core_elems(const mps_t* m, int k);
int mps_init(vp_ctx* ctx, mps_t* m, int n);
void mps_free(mps_t* m);
bool xdesc(const vp_layout* L);        // x bits fine to coarse (S2)
bool vdesc(const vp_layout* L);        // v bits fine to coarse (S3)
bool interleaved(const vp_layout* L);  // IF or IG
bool grouped(const vp_layout* L);      // IG
bool layout_ok(const vp_layout* L);
std::vector<int> site_dims(const vp_layout* L);  // per site: 0 = x bit, 1 = v bit
double grid_dx(const vp_layout* L);
double grid_dv(const vp_layout* L);

}  // namespace vp

struct vp_sim {
  vp_ctx* ctx = nullptr;
  vp_layout lay{};
  vp_config cfg{};
  std::vector<int> dims;
  mps_t f, fi, acc, wa, wb, em;
  mps_t kd, ku, kt;              // derivative and its two terms (levels C4, C5)
  mpo_t LT;                      // field term alone (level C5)
  vp::Chain U;                       // static upwind part (host copy, for bonds)
  std::vector<vp::DevBuf> Ud;        // device cores of U
  vp::Chain Dv;                      // zero-gradient v derivative chain
  std::vector<vp::DevBuf> Dvd;
  mpo_t L;                       // operator of the current stage
  vp::DevBuf rho, E, evec;
  double t = 0.0;
  vp::Flops flops;
  std::vector<double> entropy;  // per-bond EE of the last final compression
  vp_ctx* ctxB = nullptr;  // second stream: the f_{i+1} compressions run beside the acc ones
  cudaEvent_t evA = nullptr, evB = nullptr;
  double ecoef = 1.0;      // -q/m of the species: the field term is diag(ecoef E) (x) D_v
  int coop_div = 1;        // runs sharing the GPU at once: grid-cooperative QRs get num_sms / (2 coop_div)
  vp_group* lockstep = nullptr;  // cfg.streams == 0: the one-member group that steps this sim
};

namespace vp {
// A sim whose configuration the lockstep group steps: compression level C1,
// the plain sweeps, FP64 or FP32 contractions, tolerances >= 1e-13, one
// species against a fixed background.
bool lockstep_eligible(const vp_sim* s);
}  // namespace vp
