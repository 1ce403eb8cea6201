// Host side of the persistent step kernel (k_persist.cuh): shared memory,
// grid size, launch; the register budget of 3 CTAs per SM is instantiated
// here, the 4-per-SM FP32 one for batches in k_persist_wide.cu.
#include "k_persist.cuh"

namespace phd {

void* persist_kernel_wide_f32(int rb);   // k_persist_wide.cu

// Dynamic shared memory of the kernel for a handle's m_max (the largest of
// the phases' layouts).
template <class R> size_t persist_smem(int m_max) {
  const size_t mm = ((size_t)m_max + 7) & ~(size_t)7;
  const size_t a = 16 * kCells * sizeof(int);                                        // D
  const size_t l = (kPT / 32) * sizeof(unsigned long long) + kGT * (sizeof(int) + sizeof(St4<R>));  // L
  const size_t e = kGT * sizeof(P4<R>) + mm * sizeof(int);                          // E
  const size_t g = mm * (sizeof(int) + sizeof(Z4<R>)) + (kPT / 32) * mm * sizeof(unsigned short);   // G
  const size_t j = kGT * sizeof(P4<R>) + kGT * sizeof(St4<R>) + mm * sizeof(int2) + mm * sizeof(int);  // J
  size_t s = a;
  if (e > s) s = e;
  if (g > s) s = g;
  if (j > s) s = j;
  if (l > s) s = l;
  return (s + 127) & ~(size_t)127;
}

template <class R, int RB> static void* persist_fn() { return reinterpret_cast<void*>(&k_step_grid<R, RB, 3>); }

// the kernel for a handle: batches (wide) in FP32 take the 4-per-SM budget
template <class R> static void* persist_kernel(int rb, bool wide) {
  if (wide && sizeof(R) == 4) return persist_kernel_wide_f32(rb);
  switch (rb) {
    case 1: return persist_fn<R, 1>();
    case 2: return persist_fn<R, 2>();
    case 3: return persist_fn<R, 3>();
    default: return persist_fn<R, 0>();
  }
}

// CTAs of the cooperative launch: co-resident blocks per SM x SMs (0 if the
// kernel cannot be launched with this shared memory).
template <class R> int persist_grid(const Model& m, bool wide) {
  void* fn = persist_kernel<R>(model_flag(m), wide);
  const size_t smem = persist_smem<R>(m.m_max);
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kPT, smem) != cudaSuccess) return 0;
  if (per > 4) per = 4;
  return per * sms;
}

template <class R>
cudaError_t launch_persist(const Dev& d, const Model& m, int grid, const R* Z, int M, const R* noise,
                           const uint32_t* u, R* out_states, int* out_labels, int cap, int* d_count,
                           unsigned long long base, bool direct, bool advance, cudaStream_t s) {
  PersistArgs<R> a{Z, M, noise, u, out_states, out_labels, cap, d_count, base, direct ? 1 : 0, advance ? 1 : 0};
  Dev dd = d;
  Model mm = m;
  void* args[] = {&dd, &mm, &a};
  return cudaLaunchCooperativeKernel(persist_kernel<R>(model_flag(m), !direct), dim3(grid), dim3(kPT), args,
                                     persist_smem<R>(m.m_max), s);
}

// barriers after A, C, D, E, F, G, (H: batches and PEs), J, K
int persist_barriers(bool direct) { return direct ? 8 : 9; }

template size_t persist_smem<float>(int);
template size_t persist_smem<double>(int);
template int persist_grid<float>(const Model&, bool);
template int persist_grid<double>(const Model&, bool);
template cudaError_t launch_persist<float>(const Dev&, const Model&, int, const float*, int, const float*,
                                           const uint32_t*, float*, int*, int, int*, unsigned long long, bool,
                                           bool, cudaStream_t);
template cudaError_t launch_persist<double>(const Dev&, const Model&, int, const double*, int, const double*,
                                            const uint32_t*, double*, int*, int, int*, unsigned long long, bool,
                                            bool, cudaStream_t);

}  // namespace phd
