// gl_internal.h - helpers shared between the library's translation units (not ABI).
#pragma once

#include <cuda_runtime.h>

#include "gl_device.cuh"
#include "gl_launch.h"

struct gl_system;

namespace gl_internal {

// GL_OK if sys lives on the current device, else GL_ERR_INVALID_ARG (message set).
int system_device_check(const gl_system* s);

// Device bytes of likelihood scratch the system holds now (grown on demand).
size_t scratch_held(const gl_system* s);

// Segment of a call on sys (system data, tile plan) with null scratch pointers.
gl::Seg seg_without_scratch(const gl_system* s, const float* params, int B);

// Record the calling thread's error message and return code.
int set_error(int code, const char* msg);
int cuda_error(cudaError_t e, const char* what);

// Launch hooks of the library (launch counting, optional event timing).
gl::Hooks* hooks();

// Add kernels launched outside the hooks (graph replays) to the launch count.
void count_launches(long long n);

// The likelihood profiled over the light amplitudes (gl_variant.cu).
// With loglik set also log L and chi^2 of the profiled model and, with dldm
// set, d log L / d M per pixel ([B, H, W]).
cudaError_t launch_amp_solve(int B, int HW, const float* images, const float* data, const float* sigma2,
                             const float* params, float* params_out, double* amps, float inv_gain, double* loglik,
                             double* chi2, float* dldm, cudaStream_t st);
cudaError_t launch_zero_amp_grad(int B, double* grad, cudaStream_t st);

}  // namespace gl_internal
