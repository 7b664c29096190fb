// launch.h - every kernel launch of libmlsgd goes through launch(): it counts the
// launch and, when profiling is enabled for the kernel's class, brackets it with
// CUDA events on the launching stream and accumulates its algorithmic bytes
// (each input read once, each output written once).
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace mlsgd {

void prof_begin(const char* cls, cudaStream_t st);
void prof_end(const char* cls, cudaStream_t st, double bytes, double flops);

template <typename... KArgs, typename... Args>
inline void launch(const char* cls, double bytes, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                   cudaStream_t st, Args&&... args) {
  prof_begin(cls, st);
  kern<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
  prof_end(cls, st, bytes, 0.0);
}

template <typename... KArgs, typename... Args>
inline void launch_flops(const char* cls, double bytes, double flops, void (*kern)(KArgs...), dim3 grid, dim3 block,
                         size_t smem, cudaStream_t st, Args&&... args) {
  prof_begin(cls, st);
  kern<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
  prof_end(cls, st, bytes, flops);
}

}  // namespace mlsgd
