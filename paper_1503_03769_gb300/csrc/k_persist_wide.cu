// The persistent step kernel (k_persist.cuh) with the register budget of 4
// CTAs per SM, FP32, for batches of independent runs (its own translation
// unit, so the library's sources still compile in parallel).
#include "k_persist.cuh"

namespace phd {

void* persist_kernel_wide_f32(int rb) {
  switch (rb) {
    case 1: return reinterpret_cast<void*>(&k_step_grid<float, 1, 4>);
    case 2: return reinterpret_cast<void*>(&k_step_grid<float, 2, 4>);
    case 3: return reinterpret_cast<void*>(&k_step_grid<float, 3, 4>);
    default: return reinterpret_cast<void*>(&k_step_grid<float, 0, 4>);
  }
}

}  // namespace phd
