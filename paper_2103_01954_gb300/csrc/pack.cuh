// pack.cuh -- payload precision conversion and camera ray generation.
#pragma once

#include "common.cuh"

namespace mvp {

struct Cam {
  float m[12];  // row-major 3x4 [right down forward | eye]
  float focal;
  int width, height;
};

cudaError_t launch_pack(const float *src, void *dst, int64_t n, int dtype, cudaStream_t st);
cudaError_t launch_camera(const Cam &c, float *o, float *d, cudaStream_t st);

}  // namespace mvp
