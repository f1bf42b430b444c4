// vp_adjoint.cuh -- host interface of the functional-adjoint kernels.
#pragma once
#include <string>

#include "../../include/vpath.h"
#include "vp_cvpair.cuh"

namespace vp {

struct AdjInput {
  const double *frames;  // host [n_frames][3 n_cv]
  int n_frames, n_cv, min_sep, n_tiles;
  const int2 *tiles;     // device: the system's CV tiles
  const double *cnat;    // device: the system's C~_nat table
  const double *gm;      // device: gamma_i m_i of the system's atoms
  float L, iL;
  double zconst;         // sum of C~_nat^2
  CvConst k;
  double c;              // dt (k_R/2)^2
  const double *coef;    // host [2 n_frames] (A_n, B_n) or NULL: from the frames (z_m starts at frame 0)
  double *phi, *z_out, *Q_out, *grad;  // host outputs (may be NULL)
};

int adjoint_frames(const AdjInput &in, cudaStream_t st, std::string &err);
int adjoint_coefficients(const double *z, const double *Q, int n, double c, double *coef, double *phi,
                         cudaStream_t st, std::string &err);
// descent on Phi over frames 1 .. n_frames-2 (in.frames is ignored; frames is
// read and overwritten), Armijo backtracking; phi_hist[n_iter + 1]
int refine_frames(const AdjInput &in, double *frames, int n_iter, double step, double *phi_hist, int *n_accepted,
                  cudaStream_t st, std::string &err);

}  // namespace vp
