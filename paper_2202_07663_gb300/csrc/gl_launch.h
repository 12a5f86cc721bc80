// gl_launch.h - host-side launch interface between the C ABI and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "../../include/gigalens.h"

namespace gl {

struct Seg;

// MODE_CORR: the vectors' d log L / d M is already in their work slots (set by
// the caller); the launch runs the per-vector setup, the PSF correlation and
// the ray adjoint only (gradient without a forward pass).
enum Mode { MODE_SIM = 0, MODE_LOGLIK = 1, MODE_GRAD = 2, MODE_CORR = 3 };

// Called around every kernel launch: instrumentation and error checks.
struct Hooks {
  virtual void before(int kind, cudaStream_t st) = 0;
  virtual cudaError_t after(int kind, cudaStream_t st) = 0;
  virtual ~Hooks() = default;
};

// Dynamic shared memory of the convolution stage for an H x W image, K x K
// PSF, with or without the second buffer that keeps the pixel adjoint on chip.
size_t conv_smem_bytes(int H, int W, int K, bool two_buf);

// Largest dynamic shared memory for which the second buffer is used.
constexpr size_t CONV_TWO_BUF_MAX_SMEM = 200 * 1024;

// Above this dynamic shared memory a convolution block has an SM's shared
// memory (228 KB) to itself, so the PSF classes with a compile-time side run
// it with 512 threads (16 warps) instead of 128 or 256.
constexpr size_t CONV_WIDE_MIN_SMEM = 100 * 1024;

// Whether the convolution of an H x W image, K x K PSF uses the second buffer.
bool conv_two_buf(int H, int W, int K);
// Shared memory of the separable convolution (rank-R PSF), whether a system
// of this size takes it, and the dynamic shared memory of a segment's
// convolution (separable or direct, as its flags say).
size_t conv_sep_smem_bytes(int H, int W, int K, int R);
bool conv_sep_ok(int H, int W, int K, int R);
// Whether a system of this size convolves a rank-R PSF separably in single
// calls (whole image in one block, or in row bands over a cluster).
bool conv_sep_any(int H, int W, int K, int R);
size_t seg_conv_smem(const Seg& g);

// Convolution kernel class of a PSF side (0: K = 11, 1: K = 21, 2: any other odd K).
int conv_class(int K);
constexpr int CONV_CLASSES = 3;

// One convolution launch of a grouped call: segments [first, first + nseg) of
// the (class-sorted) table, nitems vectors, dynamic shared memory smem.
struct ConvRun {
  int cls, first, nseg, nitems;
  size_t smem;
};

// Split each vector's detector pixels into ray tiles for a batch of B.
void plan_tiles(int B, int H, int W, int k, int* ntiles, int* tile_pix);

// One segment, passed by value.
cudaError_t launch_one(const Seg& s, int mode, cudaStream_t st, Hooks* hooks);

// Basis images of the likelihood profiled over the light amplitudes: for the
// s.B vectors, the PSF-convolved lens light at I_l = 1 into s.sim[2b] and the
// lensed source light at I_s = 1 into s.sim[2b + 1] (one ray pass; s.work
// needs 2 s.B image slots).
cudaError_t launch_basis(const Seg& s, cudaStream_t st, Hooks* hooks);

// Segments in device memory, sorted by convolution class (grouped launch;
// persistent grids); one convolution launch per ConvRun.
cudaError_t launch_table(const Seg* d_segs, int nseg, int vec_total, int ray_total, const ConvRun* conv, int nconv,
                         int mode, cudaStream_t st, Hooks* hooks);

struct TableHdr;

// Set the kernel attributes a launch_devtable with these shared-memory sizes
// needs (call before capturing it).
cudaError_t prepare_devtable(const size_t* conv_smem);

// Grouped launch reading its item counts from device memory (graph-capturable).
cudaError_t launch_devtable(const TableHdr* d_hdr, const Seg* d_segs, const size_t* conv_smem, cudaStream_t st,
                            Hooks* hooks);

// Kernels launched by one launch_devtable call.
constexpr int DEVTABLE_LAUNCHES = 4 + CONV_CLASSES;

}  // namespace gl
