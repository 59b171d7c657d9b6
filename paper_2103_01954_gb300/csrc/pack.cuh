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
// decode-side epilogues (decode.cu)
cudaError_t launch_fade(const float *src, void *dst, int64_t n_prims, int M, int dtype, float alpha, int beta,
                        cudaStream_t st);
cudaError_t launch_assemble(const float *rgb, const float *op, void *dst, int64_t n_prims, int M, int dtype,
                            float alpha, int beta, cudaStream_t st);
cudaError_t launch_aa_to_quat(const float *r, int n, float *q, cudaStream_t st);
cudaError_t launch_aa_vjp(const float *r, const float *gq, int n, float *gr, cudaStream_t st);
cudaError_t launch_volume_prior(const float *s, int n, float lambda, float *loss, float *gs, cudaStream_t st);

}  // namespace mvp
