// camera.cuh -- pinhole ray of one pixel, shared by mvp_camera_rays and the serving
// kernel so that both produce the same rays bit for bit (explicit rounding).
#pragma once

#include "common.cuh"

namespace mvp {

// c2w: row-major 3x4 [right down forward | eye]; pixel centre (col + 0.5, row + 0.5),
// principal point at the image centre, focal f in pixels; d is normalised.
__device__ __forceinline__ void camera_ray(const float *m, float f, int width, int height, int row, int col,
                                           float o[3], float d[3]) {
  float cx = __fdiv_rn(__fsub_rn(__fadd_rn((float)col, 0.5f), __fmul_rn(0.5f, (float)width)), f);
  float cy = __fdiv_rn(__fsub_rn(__fadd_rn((float)row, 0.5f), __fmul_rn(0.5f, (float)height)), f);
  float dx = __fadd_rn(__fmaf_rn(m[1], cy, __fmul_rn(m[0], cx)), m[2]);
  float dy = __fadd_rn(__fmaf_rn(m[5], cy, __fmul_rn(m[4], cx)), m[6]);
  float dz = __fadd_rn(__fmaf_rn(m[9], cy, __fmul_rn(m[8], cx)), m[10]);
  float n2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
  float inv = __fdiv_rn(1.0f, __fsqrt_rn(n2));
  o[0] = m[3];
  o[1] = m[7];
  o[2] = m[11];
  d[0] = __fmul_rn(dx, inv);
  d[1] = __fmul_rn(dy, inv);
  d[2] = __fmul_rn(dz, inv);
}

}  // namespace mvp
