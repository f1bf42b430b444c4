// vp_contacts.cuh -- device view of the native-contact formation tracker.
#pragma once
#include "vp_dev.cuh"

namespace vp {

struct ContactDev {
  int32_t every = 0;               // check period in steps (0: off)
  int32_t max_nc = 0;              // most native contacts of any system
  const int2 *pairs = nullptr;     // native contacts (i, j) of every system, concatenated
  const int32_t *sys_off = nullptr, *sys_n = nullptr;  // per system: first pair, count
  const int32_t *trial_sys = nullptr;                  // per trial: its system
  long long *t = nullptr;          // per trial and contact: formation step (-1: not formed)
  const long long *t_off = nullptr;                    // per trial: first entry in t
  float r2_lo = 0.f, r2_hi = 0.f;  // FP32 guard band around the formation threshold r_h^2
  double r0 = 0.0;                 // contact radius of C(r)
};

void launch_contacts(const Dev &d, const ContactDev &c, cudaStream_t s);

}  // namespace vp
