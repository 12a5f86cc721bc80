// gl_kernels.cu - sm_103a kernels of the batched lens likelihood and gradient.
//
// Launch sequence of one call (arXiv:2202.07663, Sec. 2.1.1 -> 2.1.2 -> 2.2):
//   k_setup    per vector: FP64 derived constants (ellipticity forms, series
//              coefficients, Sersic exponents) -> VecConst
//   k_ray_fwd  per (vector, pixel tile): k x k rays per detector pixel, EPL +
//              shear deflection, source and lens Sersic, k x k mean -> work
//   k_conv     per vector: shared-memory PSF convolution of work, per-pixel
//              Gaussian log-likelihood term, FP64 block reduction -> log L;
//              for the gradient also the pixel adjoint d log L / d I_model,
//              correlated with the PSF and divided by k^2 -> work
//   k_ray_adj  per (vector, pixel tile): rays recomputed, forward-mode
//              derivatives contracted with the subpixel adjoint -> partial
//   k_final    per vector: fixed-order FP64 sum of the tile partials and the
//              per-vector chain rule -> grad
// Every kernel loops over its items with a grid stride, so the same code
// serves one-system launches (one segment passed by value) and grouped
// launches over many systems (segment table in device memory).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <atomic>
#include <map>
#include <mutex>
#include <type_traits>

#include "gl_device.cuh"
#include "gl_launch.h"

namespace gl {

// ------------------------------------------------------ segment sources ---

struct OneSeg {
  Seg s;
  __device__ __forceinline__ int nvec() const { return s.B; }
  __device__ __forceinline__ int nray() const { return s.B * s.ntiles; }
  __device__ __forceinline__ int nconv() const { return s.B; }
  __device__ __forceinline__ const Seg* vec_seg(int item, int& local) const { local = item; return &s; }
  __device__ __forceinline__ const Seg* ray_seg(int item, int& local) const { local = item; return &s; }
  __device__ __forceinline__ const Seg* conv_seg(int item, int& local) const { local = item; return &s; }
};

// Segments in device memory. The convolution kernel of one PSF class sees
// the contiguous run [conv_first, conv_first + conv_nseg) of the table.
struct SegTable {
  const Seg* segs;   // device, sorted by PSF class, then vec_begin / ray_begin ascending
  int nseg, vec_total, ray_total;
  int conv_first, conv_nseg, conv_total;
  __device__ __forceinline__ int nvec() const { return vec_total; }
  __device__ __forceinline__ int nray() const { return ray_total; }
  __device__ __forceinline__ int nconv() const { return conv_total; }
  __device__ __forceinline__ const Seg* conv_seg(int item, int& local) const {
    const Seg* c = segs + conv_first;
    int lo = 0;
    for (int i = 1; i < conv_nseg; ++i) lo = (c[i].conv_begin <= item) ? i : lo;
    local = item - c[lo].conv_begin;
    return c + lo;
  }
  __device__ __forceinline__ const Seg* vec_seg(int item, int& local) const {
    int lo = 0;
    for (int i = 1; i < nseg; ++i) lo = (segs[i].vec_begin <= item) ? i : lo;
    local = item - segs[lo].vec_begin;
    return segs + lo;
  }
  __device__ __forceinline__ const Seg* ray_seg(int item, int& local) const {
    int lo = 0;
    for (int i = 1; i < nseg; ++i) lo = (segs[i].ray_begin <= item) ? i : lo;
    local = item - segs[lo].ray_begin;
    return segs + lo;
  }
};

// Segment table and item counts in device memory, read when the kernels run,
// so that one captured graph serves every batch composition.
struct DevTable {
  const TableHdr* hdr;
  const Seg* segs;     // sorted by PSF class, then vec_begin / ray_begin ascending
  int cls;             // convolution class of this launch (conv kernel only)
  __device__ __forceinline__ int nvec() const { return hdr->vec_total; }
  __device__ __forceinline__ int nray() const { return hdr->ray_total; }
  __device__ __forceinline__ int nconv() const { return hdr->conv_total[cls]; }
  __device__ __forceinline__ const Seg* vec_seg(int item, int& local) const {
    const int n = hdr->nseg;
    int lo = 0;
    for (int i = 1; i < n; ++i) lo = (segs[i].vec_begin <= item) ? i : lo;
    local = item - segs[lo].vec_begin;
    return segs + lo;
  }
  __device__ __forceinline__ const Seg* ray_seg(int item, int& local) const {
    const int n = hdr->nseg;
    int lo = 0;
    for (int i = 1; i < n; ++i) lo = (segs[i].ray_begin <= item) ? i : lo;
    local = item - segs[lo].ray_begin;
    return segs + lo;
  }
  __device__ __forceinline__ const Seg* conv_seg(int item, int& local) const {
    const Seg* c = segs + hdr->conv_first[cls];
    const int n = hdr->conv_nseg[cls];
    int lo = 0;
    for (int i = 1; i < n; ++i) lo = (c[i].conv_begin <= item) ? i : lo;
    local = item - c[lo].conv_begin;
    return c + lo;
  }
};

// Copy a struct of 4-byte words into shared memory with the whole block.
template <class T>
__device__ __forceinline__ void block_copy(T* dst, const T* src) {
  static_assert(sizeof(T) % 4 == 0, "word copy");
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < int(sizeof(T) / 4); i += blockDim.x) d[i] = s[i];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-vector constants live in slots. With ray_order, k_order has put the
// vectors in the slots longest EPL series first, and k_setup writes into
// each slot the vector it holds (VecConst::order); else slot p holds vector
// p. The ray kernels take their items slot by slot, so the heaviest
// vectors' blocks come first, and write every result at the vector's own
// index.
// A slot's vector outside 0 .. B - 1 can only come from parameters changed
// by another stream while k_order ran; it is then read as p, so that no
// access leaves the batch.
__device__ __forceinline__ int slot_checked(int o, int p, int B) { return unsigned(o) < unsigned(B) ? o : p; }
__device__ __forceinline__ int slot_vector(const Seg& s, int p) {
  return s.ray_order ? slot_checked(s.vc[p].order, p, s.B) : p;
}
// The same in k_setup, from the slot array k_order left at the start of the
// work buffer (work + B ints).
__device__ __forceinline__ int setup_vector(const Seg& s, int p) {
  return s.ray_order ? slot_checked(reinterpret_cast<const int*>(s.work)[s.B + p], p, s.B) : p;
}

// Slot q and tile of a segment's ray item (local index in the segment); the
// items of one slot are consecutive.
__device__ __forceinline__ void ray_item(const Seg& ss, int local, int& q, int& tile) {
  q = local / ss.ntiles;
  tile = local - q * ss.ntiles;
}

// ------------------------------------------------------------- k_setup ----

// Derived constants of one Sersic profile (R_eff, n, e1, e2, xc, yc, I0),
// formed in FP64 and rounded once: each is the same for every ray, so its
// rounding acts like a change of the parameters. 1/R_eff^2 is folded into
// the quadratic form (R_eff^2 floored at 1e-30 so that no coefficient
// overflows). One FP64 division. Validity (R > 0, n > 0, |e| < 1) is
// checked elsewhere.
__device__ void setup_light(const float* p, LightC& L) {
  const float R = p[0], n = p[1];
  const double d1 = p[2], d2 = p[3], dn = n;
  const double e2s = d1 * d1 + d2 * d2;
  const double R2 = fmax(double(R) * double(R), 1e-30), om = 1.0 - e2s;
  const double iDR = 1.0 / (om * R2);        // 1 / ((1 - e^2) R^2)
  const double iD2R = iDR * iDR * R2;        // 1 / ((1 - e^2)^2 R^2)
  L.A = float((1.0 + e2s - 2.0 * d1) * iDR);
  L.B2 = float(-4.0 * d2 * iDR);
  L.C = float((1.0 + e2s + 2.0 * d1) * iDR);
  L.x = p[4];
  L.y = p[5];
  L.c1 = __fdiv_rn(0.5f, n);                 // one rounding, as in FP64
  L.r2min = float(double(RHO2_MIN) * om * iDR);
  L.k1 = float((1.9992 * dn - 0.3271) * 1.4426950408889634074);   // b_n / ln 2
  L.I0 = p[6];
  // derivatives of (A, 2B, C) with respect to e1 and e2
  L.A1 = float(2.0 * (d2 * d2 - (1.0 - d1) * (1.0 - d1)) * iD2R);
  L.B21 = float(-8.0 * d1 * d2 * iD2R);
  L.C1 = float(2.0 * ((1.0 + d1) * (1.0 + d1) - d2 * d2) * iD2R);
  L.A2 = float(4.0 * d2 * (1.0 - d1) * iD2R);
  L.B22 = float(-4.0 * (1.0 - d1 * d1 + d2 * d2) * iD2R);
  L.C2 = float(4.0 * d2 * (1.0 + d1) * iD2R);
}

// The FP64-formed constants of one vector, part 0 the EPL (log2(thetaE /
// rho) = lc - log2(|w|^2)/2 with lc = log2(thetaE sqrt(1 - |eps|^2)) as a
// rounded float plus t x its rounding error), parts 1 and 2 the two light
// profiles. GB300's FP64 pipe is narrow, so k_setup gives these to
// different lanes of one warp, several vectors per warp.
template <class Src>
__device__ void setup_fp64_part(const Src& src, int item, int part) {
  int p;
  const Seg* s = src.vec_seg(item, p);
  VecConst* V = s->vc + p;
  const float* pp = s->params + size_t(setup_vector(*s, p)) * NPARAM;
  if (part == 0) {
    const double e1 = pp[2], e2 = pp[3], thetaE = pp[0];
    const double om = 1.0 - (e1 * e1 + e2 * e2);
    const double lc = 0.5 * log2(thetaE * thetaE * om);
    V->lc = float(lc);
    V->tlc_lo = float((double(pp[1]) - 1.0) * (lc - double(float(lc))));
    V->w2min = float(double(RHO2_MIN) * om);
  } else {
    LightC L;
    setup_light(pp + (part == 1 ? 8 : 15), L);
    V->light[part - 1] = L;
  }
}

// Truncation target of the EPL series F = sum a_n u^n, |u| = f, a_n = c_1 ... c_n:
// the smallest N with |a_{N+1}| f^(N+1) / (1 - f max(1, c_{N+2})) <= SERIES_TOL,
// a bound on |F - F_N| (|c_k| decreases toward 1 for k >= 2, so the tail after
// a_{N+1} is at most a geometric series of ratio f max(1, c_{N+2})). The
// adjoint uses the same N (at least 1): its dF/du comes from F and h_1 in
// closed form, and the tail of dF/dt exceeds that of F only by a logarithmic
// factor.
constexpr double SERIES_TOL = 2e-8;

__device__ __forceinline__ float series_coef(int k, float t) { return (2.f * k - 2.f + t) / (2.f * k + 2.f - t); }
__device__ __forceinline__ float series_dcoef(int k, float t) {   // d c_k / d t = 4k / (2k + 2 - t)^2
  const float iden = 1.0f / (2.f * k + 2.f - t);
  return 4.f * k * iden * iden;
}

// Term count over the first NC chunks of 32 candidates (NMAX if none of them
// qualifies): lane tests N = lane + 32 m, with log|a_{N+1}| from a warp prefix
// sum of log|c_k| (k = lane + 1 + 32 m). The first chunk's result does not
// depend on NC.
template <int NC>
__device__ __forceinline__ int term_count(int lane, float t, float f, float lf, float ltol) {
  float la[NC];
#pragma unroll
  for (int m = 0; m < NC; ++m) la[m] = logf(fabsf(series_coef(lane + 1 + 32 * m, t)));
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const float y = __shfl_up_sync(0xffffffffu, la[m], o);
      if (lane >= o) la[m] += y;
    }
  }
  float carry = 0.f;
#pragma unroll
  for (int m = 0; m < NC; ++m) {
    la[m] += carry;
    carry = __shfl_sync(0xffffffffu, la[m], 31);
  }
  int n = NMAX;
#pragma unroll
  for (int m = NC - 1; m >= 0; --m) {
    const int N = lane + 32 * m;
    const float r = fminf(f * fmaxf(1.f, series_coef(N + 2, t)), 0.999999f);
    const unsigned ok_m = __ballot_sync(0xffffffffu, la[m] + (N + 1) * lf - log1pf(-r) <= ltol);
    if (ok_m) n = 32 * m + __ffs(ok_m) - 1;
  }
  return n;
}

// a_n = c_1 ... c_n and d a_n / d t for n <= 32 NC by a warp scan of the pairs
// (c_k, d c_k / d t) under (x1, y1) (x2, y2) = (x1 x2, x1 y2 + x2 y1) (the
// product rule); the first chunk's values do not depend on NC.
template <int NC>
__device__ __forceinline__ void series_coeffs(int lane, float t, VecConst* V) {
  float xs[NC], ys[NC];
#pragma unroll
  for (int m = 0; m < NC; ++m) {
    xs[m] = series_coef(lane + 1 + 32 * m, t);
    ys[m] = series_dcoef(lane + 1 + 32 * m, t);
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const float px = __shfl_up_sync(0xffffffffu, xs[m], o), py = __shfl_up_sync(0xffffffffu, ys[m], o);
      if (lane >= o) {
        ys[m] = fmaf(px, ys[m], xs[m] * py);
        xs[m] = px * xs[m];
      }
    }
  }
  float tx = 1.f, ty = 0.f;   // the product over the earlier chunks
#pragma unroll
  for (int m = 0; m < NC; ++m) {
    const float x = tx * xs[m], y = fmaf(tx, ys[m], xs[m] * ty);
    V->an[lane + 32 * m] = x;
    V->ant[lane + 32 * m] = y;
    tx = __shfl_sync(0xffffffffu, x, 31);
    ty = __shfl_sync(0xffffffffu, y, 31);
  }
}

// Block size of k_setup: eight warps of per-vector work and two for the
// FP64 constants of their vectors.
constexpr int SETUP_THREADS = 10 * 32;

// A block takes its vectors wpb (warps per block less two) at a time. The
// last two warps form the FP64 constants (setup_fp64_part): the first of
// them the EPL part of each vector (lane v), the second the two light
// profiles (lane 2 v + part - 1), so that neither warp's lanes diverge
// between the two code paths and one warp's FP64 instructions serve several
// vectors. Each other warp takes one vector: lanes 0..21 check one
// parameter each, lane 0 the EPL's FP32 constants, lanes 1 and 2 the
// validity of the light profiles; all lanes compute the series coefficients
// and, by ballot, the term count (FP32: every constant feeds FP32
// arithmetic). The kinds of warp run side by side and write disjoint fields
// of VecConst (one call at 60x60, B = 4096: 12.5 -> 11.8 us against the
// FP64 parts in the first warp before its own vector).
template <class Src>
__global__ void k_setup(const __grid_constant__ Src src) {
  const PdlScope pdl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wpb = (blockDim.x >> 5) - 2;
  const int nvec = src.nvec();
  for (int base = blockIdx.x * wpb; base < nvec; base += gridDim.x * wpb) {
    if (warp >= wpb) {
      const bool epl = warp == wpb;
      const int v = epl ? lane : lane >> 1;
      if (v < wpb && base + v < nvec) setup_fp64_part(src, base + v, epl ? 0 : 1 + (lane & 1));
      continue;
    }
    const int item = base + warp;
    if (item >= nvec) continue;   // warp-uniform
    int p;
    const Seg* s = src.vec_seg(item, p);
    VecConst* V = s->vc + p;
    const int b = setup_vector(*s, p);
    const float* pp = s->params + size_t(b) * NPARAM;
    bool ok = lane >= NPARAM || isfinite(pp[lane]);
    const float e1 = pp[2], e2 = pp[3], t = pp[1] - 1.0f;
    const float e2s = fmaf(e1, e1, e2 * e2);
    if (lane == 0) {
      V->order = b;
      const float thetaE = pp[0];
      ok = ok && thetaE > 0.f && e2s < 1.f && t > -1.f && t < 3.f;
      const float i1me2 = 1.0f / (1.0f - e2s);
      V->xc = pp[4];
      V->yc = pp[5];
      V->e1 = e1;
      V->e2 = e2;
      V->t = t;
      V->g1 = pp[6];
      V->g2 = pp[7];
      V->th = 0.5f * t;
      V->kc = 1.f - 0.5f * t;
      V->kap_c = 0.5f * (2.f - t);
      V->omt = 1.f - t;
      V->e1i = e1 * i1me2;
      V->e2i = e2 * i1me2;
    } else if (lane == 1 || lane == 2) {
      const float* lp = pp + (lane == 1 ? 8 : 15);
      ok = ok && lp[0] > 0.f && lp[1] > 0.f && fmaf(lp[2], lp[2], lp[3] * lp[3]) < 1.f;
    }
    ok = __all_sync(0xffffffffu, ok);
    // term count and coefficients over the first 32 candidates; the other
    // chunks only for the vectors (large |eps|) whose series is longer
    const float f = sqrtf(e2s);
    const float lf = f > 0.f ? logf(f) : -1e30f;
    const float ltol = logf(float(SERIES_TOL));
    int n_fwd = term_count<1>(lane, t, f, lf, ltol);
    if (n_fwd < 32) {   // warp-uniform
      series_coeffs<1>(lane, t, V);
    } else {
      n_fwd = term_count<NMAX / 32>(lane, t, f, lf, ltol);
      series_coeffs<NMAX / 32>(lane, t, V);
    }
    if (lane == 0) {
      V->nterms = ok ? min(n_fwd, NMAX) : -1;
      V->nterms_adj = max(min(n_fwd, NMAX), 1);
    }
  }
}

// ------------------------------------------------------------- k_order ----

// Slots of a call's vectors, longest EPL series first (the order the ray
// kernels then take them in). A ray's cost grows with the vector's series
// terms N (331 + 14 N flops in the adjoint, 90 + 7 N in the forward), and a
// batch drawn from a prior mixes short and long series; with the heaviest
// vectors' blocks in the first waves the last waves hold the lightest
// (longest-processing-time first). The order is fixed before k_setup, so its
// key comes from the parameters: the series' terms fall like |eps|^n, so N
// grows like log(tol) / log|eps|, and the key is 204.8 / -log2(|eps|^2)
// (about four keys per term at tol = 2e-8), capped at NMAX - 1.
//
// Two kernels, both before k_setup, using the start of the work buffer
// (which k_ray_fwd fills only later) as int arrays: key[B], then slot[B],
// the vector each slot holds. k_keys forms the keys over many blocks (one
// block reading every vector's row of parameters waits on one SM's
// scattered loads: 11.8 us at B = 4096). k_order, one block, is a counting
// sort: each warp counts its vectors per key in a row of its own (shared-
// memory atomics that never meet another warp's: a batch's keys crowd into
// a few values, and one counter per key for the whole block would make the
// warps wait on each other), a block-wide scan over (key from the largest down, warp)
// turns the counts into first slots, and each warp hands out its slots.
// Within one (key, warp) the slots follow the order the warp's atomics are
// served in; results do not depend on the slots. k_setup reads its slot's
// vector from slot[] and keeps it in VecConst::order for the later kernels.
constexpr int KEYS_THREADS = 256;
constexpr int ORDER_THREADS = 1024;
constexpr int ORDER_WARPS = ORDER_THREADS / 32;
constexpr int ORDER_UNROLL = 4;         // keys loaded per thread before they are counted
constexpr int ORDER_PITCH = NMAX + 1;   // per-warp row of counts; the odd pitch spreads the banks
constexpr int ORDER_STAGE = 4096;       // batches up to this size are scattered in shared memory
static_assert(4 * ORDER_THREADS == ORDER_WARPS * NMAX, "the scan gives each thread four (key, warp) counts");

__device__ __forceinline__ int order_key(const float* params, int b) {
  const float e1 = params[size_t(b) * NPARAM + 2], e2 = params[size_t(b) * NPARAM + 3];
  const float e2s = fmaf(e1, e1, e2 * e2);
  if (!(e2s < 1.f)) return 0;   // NaN or |eps| >= 1 (invalid: no ray work)
  const float r = 204.8f / -lg2(e2s);   // 0 at eps = 0 (lg2 gives -inf)
  return r < float(NMAX - 1) ? int(r) : NMAX - 1;
}

__device__ __forceinline__ int* order_keys(const Seg& s) { return reinterpret_cast<int*>(s.work); }
__device__ __forceinline__ int* order_slots(const Seg& s) { return reinterpret_cast<int*>(s.work) + s.B; }

__global__ void __launch_bounds__(KEYS_THREADS) k_keys(const __grid_constant__ OneSeg src) {
  const PdlScope pdl;
  const Seg& s = src.s;
  int* key = order_keys(s);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < s.B; b += gridDim.x * blockDim.x) key[b] = order_key(s.params, b);
}

// This lane's entry of row[key], the warp's own row (key < 0: no vector):
// a shared-memory atomic that meets only the warp's other lanes.
__device__ __forceinline__ int order_take(int* row, int key) { return key >= 0 ? atomicAdd(&row[key], 1) : 0; }

__device__ __forceinline__ int order_key_at(const int* key, int b, int B) {
  if (b >= B) return -1;
  const int k = key[b];
  return k < 0 ? 0 : (k > NMAX - 1 ? NMAX - 1 : k);
}

__global__ void __launch_bounds__(ORDER_THREADS) k_order(const __grid_constant__ OneSeg src) {
  __shared__ int cnt[ORDER_WARPS * ORDER_PITCH];   // [warp][key]: vectors, then the warp's next slot
  __shared__ int wsum[ORDER_WARPS];
  __shared__ int stage[ORDER_STAGE];               // slot -> vector, for B <= ORDER_STAGE
  const PdlScope pdl;
  const Seg& s = src.s;
  const int B = s.B, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int chunk = ORDER_UNROLL * ORDER_THREADS;
  const int* keys = order_keys(s);
  int* slots = order_slots(s);
  const bool staged = B <= ORDER_STAGE;
  int* row = cnt + w * ORDER_PITCH;
  for (int i = tid; i < ORDER_WARPS * ORDER_PITCH; i += ORDER_THREADS) cnt[i] = 0;
  __syncthreads();
  int first[ORDER_UNROLL];   // the first chunk's keys, kept for the scatter
  for (int b0 = tid; b0 - tid < B; b0 += chunk) {   // the same trip count for every thread
    int key[ORDER_UNROLL];
#pragma unroll
    for (int u = 0; u < ORDER_UNROLL; ++u) key[u] = order_key_at(keys, b0 + u * ORDER_THREADS, B);
#pragma unroll
    for (int u = 0; u < ORDER_UNROLL; ++u) {
      order_take(row, key[u]);
      if (b0 == tid) first[u] = key[u];
    }
  }
  __syncthreads();
  // exclusive scan in the order (key from NMAX - 1 down, warp 0 .. 31):
  // thread t takes positions 4 t .. 4 t + 3, one key and four warps
  {
    const int key = NMAX - 1 - (4 * tid) / ORDER_WARPS, w0 = (4 * tid) % ORDER_WARPS;
    int v[4], sum = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      v[j] = cnt[(w0 + j) * ORDER_PITCH + key];
      sum += v[j];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
      const int t = wsum[lane];
      int c = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, c, o);
        if (lane >= o) c += y;
      }
      wsum[lane] = c - t;
    }
    __syncthreads();
    int slot = wsum[w] + incl - sum;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      cnt[(w0 + j) * ORDER_PITCH + key] = slot;
      slot += v[j];
    }
  }
  __syncthreads();
  // the same keys as the count, so the slots handed out are exactly 0 .. B - 1
  for (int b0 = tid; b0 - tid < B; b0 += chunk) {
    int key[ORDER_UNROLL];
#pragma unroll
    for (int u = 0; u < ORDER_UNROLL; ++u) key[u] = b0 == tid ? first[u] : order_key_at(keys, b0 + u * ORDER_THREADS, B);
#pragma unroll
    for (int u = 0; u < ORDER_UNROLL; ++u) {
      const int slot = order_take(row, key[u]);
      if (key[u] >= 0 && slot < B) {
        if (staged)
          stage[slot] = b0 + u * ORDER_THREADS;
        else
          slots[slot] = b0 + u * ORDER_THREADS;
      }
    }
  }
  if (staged) {
    __syncthreads();
    for (int i = tid; i < B; i += ORDER_THREADS) slots[i] = stage[i];
  }
}

// ----------------------------------------------------------- k_ray_fwd ----

#ifndef GL_FWD_THREADS
#define GL_FWD_THREADS 128
#endif
#ifndef GL_FWD_MINB
#define GL_FWD_MINB 4
#endif
constexpr int FWD_THREADS = GL_FWD_THREADS;

template <class Src>
__global__ void __launch_bounds__(FWD_THREADS, GL_FWD_MINB) k_ray_fwd(const __grid_constant__ Src src) {
  __shared__ VecConst sv;
  __shared__ Seg ss;
  const PdlScope pdl;
  for (int item = blockIdx.x; item < src.nray(); item += gridDim.x) {
    int local;
    const Seg* segp = src.ray_seg(item, local);
    block_copy(&ss, segp);
    __syncthreads();
    int q, tile;
    ray_item(ss, local, q, tile);
    block_copy(&sv, ss.vc + q);
    __syncthreads();
    const int b = ss.ray_order ? slot_checked(sv.order, q, ss.B) : q;   // the vector in slot q
    const int HW = ss.H * ss.W, W = ss.W, k = ss.k;
    const int p0 = tile * ss.tile_pix;
    const int p1 = min(HW, p0 + ss.tile_pix);
    const float inv_k2 = 1.0f / float(k * k);
    const bool valid = sv.nterms >= 0;
    float* out = ss.work + size_t(b) * HW;
    // two pixels per thread and step (p and p + blockDim), their rays paired in f32x2
    const int stride = blockDim.x;
    for (int p = p0 + threadIdx.x; p < p1; p += 2 * stride) {
      const int q = p + stride;
      const bool has_q = q < p1;
      const int qq = has_q ? q : p;
      const int ip = p / W, jp = p - ip * W;
      const int iq = qq / W, jq = qq - iq * W;
      F2 acc = sp<F2>(0.f);
      if (valid) {
        // grid indices of the pixels' first subpixels; a subpixel step adds 2
        const F2 ny0 = {make_float2(float(2 * ip * k + ss.ny0), float(2 * iq * k + ss.ny0))};
        const F2 nx0 = {make_float2(float(2 * jp * k + ss.nx0), float(2 * jq * k + ss.nx0))};
        F2 ny = ny0;
        for (int a = 0; a < k; ++a, ny = ny + sp<F2>(2.f)) {
          const F2 y = grid_coord2(ny, ss.hh, ss.hl);
          F2 nx = nx0;
          for (int c = 0; c < k; ++c, nx = nx + sp<F2>(2.f)) {
            const F2 x = grid_coord2(nx, ss.hh, ss.hl);
            acc = acc + ray_intensity_T(sv, sv.an, x, y);
          }
        }
        acc = acc * sp<F2>(inv_k2);
      } else {
        acc = sp<F2>(__int_as_float(0x7fc00000));
      }
      out[p] = acc.v.x;
      if (has_q) out[q] = acc.v.y;
    }
    __syncthreads();
  }
}

// Unit-amplitude basis images of the likelihood profiled over the light
// amplitudes: per vector the binned lens light with I_l = 1 into work slot 2b
// and the binned, lensed source light with I_s = 1 into slot 2b + 1, from one
// ray pass (both share the rays, the source the deflection); the vector's own
// amplitudes are not used. Invalid vectors get NaN in both slots.
template <class Src>
__global__ void __launch_bounds__(FWD_THREADS, GL_FWD_MINB) k_ray_fwd_basis(const __grid_constant__ Src src) {
  __shared__ VecConst sv;
  __shared__ Seg ss;
  const PdlScope pdl;
  for (int item = blockIdx.x; item < src.nray(); item += gridDim.x) {
    int local;
    const Seg* segp = src.ray_seg(item, local);
    block_copy(&ss, segp);
    __syncthreads();
    int q, tile;
    ray_item(ss, local, q, tile);
    block_copy(&sv, ss.vc + q);
    __syncthreads();
    const int b = ss.ray_order ? slot_checked(sv.order, q, ss.B) : q;   // the vector in slot q
    if (threadIdx.x == 0) {
      sv.light[0].I0 = 1.f;
      sv.light[1].I0 = 1.f;
    }
    __syncthreads();
    const int HW = ss.H * ss.W, W = ss.W, k = ss.k;
    const int p0 = tile * ss.tile_pix;
    const int p1 = min(HW, p0 + ss.tile_pix);
    const float inv_k2 = 1.0f / float(k * k);
    const bool valid = sv.nterms >= 0;
    float* out_l = ss.work + size_t(2 * b) * HW;
    float* out_s = out_l + HW;
    const int stride = blockDim.x;
    for (int p = p0 + threadIdx.x; p < p1; p += 2 * stride) {
      const int q = p + stride;
      const bool has_q = q < p1;
      const int qq = has_q ? q : p;
      const int ip = p / W, jp = p - ip * W;
      const int iq = qq / W, jq = qq - iq * W;
      F2 acc_l = sp<F2>(0.f), acc_s = sp<F2>(0.f);
      if (valid) {
        const F2 ny0 = {make_float2(float(2 * ip * k + ss.ny0), float(2 * iq * k + ss.ny0))};
        const F2 nx0 = {make_float2(float(2 * jp * k + ss.nx0), float(2 * jq * k + ss.nx0))};
        F2 ny = ny0;
        for (int a = 0; a < k; ++a, ny = ny + sp<F2>(2.f)) {
          const F2 y = grid_coord2(ny, ss.hh, ss.hl);
          F2 nx = nx0;
          for (int c = 0; c < k; ++c, nx = nx + sp<F2>(2.f)) {
            const F2 x = grid_coord2(nx, ss.hh, ss.hl);
            F2 ax, ay;
            epl_fwd_T(sv, sv.an, x, y, ax, ay);
            const F2 bx = x - ax - fmaT(sp<F2>(sv.g1), x, sp<F2>(sv.g2) * y);
            const F2 by = y - ay - fmaT(sp<F2>(sv.g2), x, sp<F2>(-sv.g1) * y);
            acc_s = acc_s + sersic_fwd_T(sv.light[1], bx, by);
            acc_l = acc_l + sersic_fwd_T(sv.light[0], x, y);
          }
        }
        acc_l = acc_l * sp<F2>(inv_k2);
        acc_s = acc_s * sp<F2>(inv_k2);
      } else {
        acc_l = acc_s = sp<F2>(__int_as_float(0x7fc00000));
      }
      out_l[p] = acc_l.v.x;
      out_s[p] = acc_s.v.x;
      if (has_q) {
        out_l[q] = acc_l.v.y;
        out_s[q] = acc_s.v.y;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------- k_ray_adj -----

// Lens or source light: accumulates R, n (two terms), e1, e2, x, y, I0 slots
// and returns (Gx, Gy) = s I / rho^2 (A dx + B dy, B dx + C dy), so that
// dI/d(centre) = (b_n/n) (Gx, Gy) and dI/d(position) = -(b_n/n) (Gx, Gy).
// Generic in the ray type (float or a packed pair).
template <class T>
__device__ __forceinline__ void light_adj(const LightC& L, T px, T py, T g, T* acc, T& Gx, T& Gy) {
  const T dx = px - sp<T>(L.x), dy = py - sp<T>(L.y);
  const T dxx = dx * dx, dxy = dx * dy, dyy = dy * dy;
  const T r2raw = fmaT(sp<T>(L.A), dxx, fmaT(sp<T>(L.B2), dxy, sp<T>(L.C) * dyy));
  const T keep = geT(r2raw, sp<T>(L.r2min));       // 0 where the radius is floored
  const T r2 = maxT(r2raw, sp<T>(L.r2min));
  const T ls = sp<T>(L.c1) * lg2T(r2);
  const T s = ex2T(ls);
  const T e = ex2T(fmaT(sp<T>(-L.k1), s, sp<T>(L.k1)));
  const T I = sp<T>(L.I0) * e;
  const T hI = g * I;
  const T hs = hI * s;
  acc[0] = acc[0] + hs;
  acc[1] = fmaT(hI, s - sp<T>(1.f), acc[1]);
  acc[2] = fmaT(hs, ls, acc[2]);
  const T q = keep * s * I * rcpT(r2);
  const float Bh = 0.5f * L.B2;
  Gx = q * fmaT(sp<T>(L.A), dx, sp<T>(Bh) * dy);
  Gy = q * fmaT(sp<T>(Bh), dx, sp<T>(L.C) * dy);
  const T gq = g * q;
  acc[3] = fmaT(gq, fmaT(sp<T>(L.A1), dxx, fmaT(sp<T>(L.B21), dxy, sp<T>(L.C1) * dyy)), acc[3]);
  acc[4] = fmaT(gq, fmaT(sp<T>(L.A2), dxx, fmaT(sp<T>(L.B22), dxy, sp<T>(L.C2) * dyy)), acc[4]);
  acc[5] = fmaT(g, Gx, acc[5]);
  acc[6] = fmaT(g, Gy, acc[6]);
  acc[7] = fmaT(g, e, acc[7]);
}

// One ray (or a packed pair): adds g x (derivatives of its intensity) to the
// 24 accumulators. Branch-free: a ray inside rho < 1e-6 arcsec has S = 0,
// which zeroes its deflection and every EPL derivative (all carry S).
template <class T>
__device__ __forceinline__ void ray_adj(const VecConst& V, const float* an, const float* ant, T x, T y, T g, T* acc) {
  T Gx, Gy;
  light_adj(V.light[0], x, y, g, acc + A_L_R, Gx, Gy);

  // EPL deflection with the pieces of its parameter derivatives
  const T dx = x - sp<T>(V.xc), dy = y - sp<T>(V.yc);
  const T wr = fmaT(sp<T>(-V.e1), dx, fmaT(sp<T>(-V.e2), dy, dx));
  const T wi = fmaT(sp<T>(V.e1), dy, fmaT(sp<T>(-V.e2), dx, dy));
  const T w2 = fmaT(wr, wr, wi * wi);
  const T keep = geT(w2, sp<T>(V.w2min));
  const T w2c = maxT(w2, sp<T>(V.w2min));   // > 0; where it clamps, S = 0 zeroes every EPL term
  const T lrho = fmaT(sp<T>(-0.5f), lg2T(w2c), sp<T>(V.lc));  // log2(thetaE / rho)
  const T S = keep * ex2T(fmaT(sp<T>(V.t), lrho, sp<T>(V.tlc_lo)));
  const T iw2 = rcpT(w2c);
  const T nwi = -wi;
  const T vr = fmaT(wr, wr, nwi * wi) * iw2;
  const T vi = sp<T>(2.f) * wr * wi * iw2;
  const T ur = fmaT(sp<T>(-V.e1), vr, sp<T>(-V.e2) * vi);
  const T ui = fmaT(sp<T>(V.e2), vr, sp<T>(-V.e1) * vi);
  const T nui = fmaT(sp<T>(-V.e2), vr, sp<T>(V.e1) * vi);   // -ui: packed FMAs take no negated operands
  // G = sum_{n<N} a_{n+1} u^n and dG/dt by Horner; F = 1 + u G, dF/dt = u dG/dt
  T Gr = sp<T>(0.f), Gi = sp<T>(0.f), Gtr = sp<T>(0.f), Gti = sp<T>(0.f);
#pragma unroll 2
  for (int n = V.nterms_adj; n >= 1; --n) {
    const T nGr = fmaT(ur, Gr, fmaT(nui, Gi, sp<T>(an[n - 1])));
    Gi = fmaT(ur, Gi, ui * Gr);
    Gr = nGr;
    const T nGtr = fmaT(ur, Gtr, fmaT(nui, Gti, sp<T>(ant[n - 1])));
    Gti = fmaT(ur, Gti, ui * Gtr);
    Gtr = nGtr;
  }
  const T hr = fmaT(ur, Gr, fmaT(nui, Gi, sp<T>(1.f))), hi = fmaT(ur, Gi, ui * Gr);     // F
  const T tr = fmaT(ur, Gtr, nui * Gti), ti = fmaT(ur, Gti, ui * Gtr);                 // dF/dt
  // dF/du = [(t/2) F - (1 - t/2) G] / (1 - u)   (Gauss contiguous relation; G = (F - 1)/u
  // without the cancellation)
  const T nr = fmaT(sp<T>(V.th), hr, sp<T>(-V.kc) * Gr), ni = fmaT(sp<T>(V.th), hi, sp<T>(-V.kc) * Gi);
  const T dr = sp<T>(1.f) - ur;                 // 1 - u = (dr, -ui) = (dr, nui)
  const T idd = rcpT(fmaT(dr, dr, ui * ui));
  const T pr = fmaT(nr, dr, ni * nui) * idd, pi = fmaT(ni, dr, nr * ui) * idd;
  const T swr = S * wr, swi = S * wi, nswi = S * nwi;   // S w
  const T ar = fmaT(swr, hr, nswi * hi);
  const T ai = fmaT(swr, hi, swi * hr);
  // t: alpha ln(thetaE/rho) + S w dF/dt
  const T lnr = sp<T>(0.69314718f) * lrho;
  const T dtr = fmaT(ar, lnr, fmaT(swr, tr, nswi * ti));
  const T dti = fmaT(ai, lnr, fmaT(swr, ti, swi * tr));
  // e1, e2
  const T Pr = fmaT(wr, dx, nwi * dy), Pi = fmaT(wr, dy, wi * dx);   // w z
  const T a1 = sp<T>(V.t) * fmaT(Pr, iw2, sp<T>(-V.e1i));             // d ln S / d e1
  const T a2 = sp<T>(V.t) * fmaT(Pi, iw2, sp<T>(-V.e2i));             // d ln S / d e2
  const T sfr = S * hr, sfi = S * hi;                                  // S F
  const T swpr = fmaT(swr, pr, nswi * pi), swpi = fmaT(swr, pi, swi * pr);  // S w F'
  const T nswpi = -swpi, ndx = -dx, ndy = -dy, nsfi = -sfi;
  const T k1 = sp<T>(2.f) * Pi * iw2, nk1 = sp<T>(-2.f) * Pi * iw2;
  const T k2 = sp<T>(2.f) * Pr * iw2, nk2 = sp<T>(-2.f) * Pr * iw2;
  const T nvr = -vr, nvi = -vi;
  const T du1r = fmaT(nk1, ui, nvr), du1i = fmaT(k1, ur, nvi);        // du/de1 = -V + i k1 u
  const T du2r = fmaT(k2, ui, nvi), du2i = fmaT(nk2, ur, vr);         // du/de2 = iV - i k2 u
  // dw/de1 = (-dx, dy), dw/de2 = (-dy, -dx)
  const T d1r = fmaT(ar, a1, fmaT(sfr, ndx, nsfi * dy)) + fmaT(swpr, du1r, nswpi * du1i);
  const T d1i = fmaT(ai, a1, fmaT(sfr, dy, nsfi * dx)) + fmaT(swpr, du1i, swpi * du1r);
  const T d2r = fmaT(ar, a2, fmaT(sfr, ndy, sfi * dx)) + fmaT(swpr, du2r, nswpi * du2i);
  const T d2i = fmaT(ai, a2, fmaT(sfr, ndx, nsfi * dy)) + fmaT(swpr, du2i, swpi * du2r);
  // centre: kappa and shear of the EPL from homogeneity, z kappa + conj(z) gamma = (1-t) alpha
  const T kap = sp<T>(V.kap_c) * S;
  const T iz2 = rcpT(maxT(fmaT(dx, dx, dy * dy), sp<T>(1e-30f)));
  const T nkap = sp<T>(-V.kap_c) * S;
  const T Qr = fmaT(sp<T>(V.omt), ar, nkap * dx), Qi = fmaT(sp<T>(V.omt), ai, nkap * dy);
  const T gr = fmaT(Qr, dx, Qi * ndy) * iz2, gi = fmaT(Qr, dy, Qi * dx) * iz2;   // Q z / |z|^2
  // lens equation with external shear, source at beta
  const T bx = x - ar - fmaT(sp<T>(V.g1), x, sp<T>(V.g2) * y);
  const T by = y - ai - fmaT(sp<T>(V.g2), x, sp<T>(-V.g1) * y);
  light_adj(V.light[1], bx, by, g, acc + A_S_R, Gx, Gy);
  // mass: g Ghat . d alpha / d p  (times b_s/n_s in the chain rule);
  // d alpha/d xc = -(kappa + gamma), d alpha/d yc = -i (kappa - gamma)
  const T gx = g * Gx, gy = g * Gy;
  acc[A_THETAE] = fmaT(gx, ar, fmaT(gy, ai, acc[A_THETAE]));
  acc[A_T] = fmaT(gx, dtr, fmaT(gy, dti, acc[A_T]));
  acc[A_E1] = fmaT(gx, d1r, fmaT(gy, d1i, acc[A_E1]));
  acc[A_E2] = fmaT(gx, d2r, fmaT(gy, d2i, acc[A_E2]));
  acc[A_XC] = acc[A_XC] - fmaT(gx, kap + gr, gy * gi);
  acc[A_YC] = acc[A_YC] - fmaT(gx, gi, gy * (kap - gr));
  acc[A_G1] = fmaT(gx, x, fmaT(-gy, y, acc[A_G1]));
  acc[A_G2] = fmaT(gx, y, fmaT(gy, x, acc[A_G2]));
}

// Ray type of the adjoint kernel: float (one ray per thread per step) or F2
// (two pixels per step, their rays paired in packed f32x2 arithmetic), with
// its block size and minimum resident blocks.
#ifndef GL_ADJ_PAIRED
#define GL_ADJ_PAIRED 1
#endif
#ifndef GL_ADJ_THREADS
#define GL_ADJ_THREADS 128
#endif
#ifndef GL_ADJ_MINB
#define GL_ADJ_MINB 2
#endif
constexpr int ADJ_THREADS = GL_ADJ_THREADS;

__device__ __forceinline__ float lane_sum(float v) { return v; }
__device__ __forceinline__ float lane_sum(F2 v) { return v.v.x + v.v.y; }

// MINB: resident blocks per SM the registers are fitted for. Two (218
// registers, no spills) suit long ray tiles; three (168 registers, 48 bytes
// of spills) overlap more blocks' prologues and epilogues and suit short ones
// (60x60 k=2: 654 -> 637 us; 100x100 k=4 at 80K rays per tile: 1725 -> 1736 us).
template <class Src, int MINB = GL_ADJ_MINB>
__global__ void __launch_bounds__(ADJ_THREADS, MINB) k_ray_adj(const __grid_constant__ Src src) {
  using RT = typename std::conditional<GL_ADJ_PAIRED != 0, F2, float>::type;
  __shared__ VecConst sv;
  __shared__ Seg ss;
  __shared__ double red[ADJ_THREADS / 32][NACC];
  const PdlScope pdl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int item = blockIdx.x; item < src.nray(); item += gridDim.x) {
    int local;
    const Seg* segp = src.ray_seg(item, local);
    block_copy(&ss, segp);
    __syncthreads();
    int q, tile;
    ray_item(ss, local, q, tile);
    block_copy(&sv, ss.vc + q);
    __syncthreads();
    const int b = ss.ray_order ? slot_checked(sv.order, q, ss.B) : q;   // the vector in slot q
    RT acc[NACC];
#pragma unroll
    for (int a = 0; a < NACC; ++a) acc[a] = sp<RT>(0.f);
    const int HW = ss.H * ss.W, W = ss.W, k = ss.k;
    const int p0 = tile * ss.tile_pix;
    const int p1 = min(HW, p0 + ss.tile_pix);
    const float* gpre = ss.work + size_t(b) * HW;
    if (sv.nterms >= 0) {
      const int stride = blockDim.x;
#if GL_ADJ_PAIRED
      {
        // whole steps: two pixels per thread (p and p + blockDim), their rays paired in f32x2
        const int nfull = (p1 - p0) / (2 * stride);
        for (int it = 0; it < nfull; ++it) {
          const int p = p0 + 2 * stride * it + threadIdx.x, q = p + stride;
          const int ip = p / W, jp = p - ip * W;
          const int iq = q / W, jq = q - iq * W;
          const F2 g = {make_float2(gpre[p], gpre[q])};
          // (indices converted per ray here: float-stepped indices, as in the
          // forward kernel, cost this register-bound kernel spills and time)
          for (int a = 0; a < k; ++a) {
            const F2 y = {make_float2(grid_coord(2 * (ip * k + a) + ss.ny0, ss.hh, ss.hl),
                                      grid_coord(2 * (iq * k + a) + ss.ny0, ss.hh, ss.hl))};
            for (int c = 0; c < k; ++c) {
              const F2 x = {make_float2(grid_coord(2 * (jp * k + c) + ss.nx0, ss.hh, ss.hl),
                                        grid_coord(2 * (jq * k + c) + ss.nx0, ss.hh, ss.hl))};
              ray_adj(sv, sv.an, sv.ant, x, y, g, acc);
            }
          }
        }
        // the ragged end (fewer than 2 blockDim pixels): its rays two per thread and step,
        // so that every thread takes a share; an odd last ray is paired with itself at zero weight
        const int base = p0 + 2 * stride * nfull, kk = k * k;
        const int nr = (p1 - base) * kk;
        for (int r = 2 * int(threadIdx.x); r < nr; r += 2 * stride) {
          const bool has2 = r + 1 < nr;
          const int r2 = has2 ? r + 1 : r;
          const int pa = base + r / kk, sa = r - (pa - base) * kk;
          const int pb = base + r2 / kk, sb = r2 - (pb - base) * kk;
          const int ia = pa / W, ja = pa - ia * W, ib = pb / W, jb = pb - ib * W;
          const int aa = sa / k, ca = sa - aa * k, ab = sb / k, cb = sb - ab * k;
          const F2 y = {make_float2(grid_coord(2 * (ia * k + aa) + ss.ny0, ss.hh, ss.hl), grid_coord(2 * (ib * k + ab) + ss.ny0, ss.hh, ss.hl))};
          const F2 x = {make_float2(grid_coord(2 * (ja * k + ca) + ss.nx0, ss.hh, ss.hl), grid_coord(2 * (jb * k + cb) + ss.nx0, ss.hh, ss.hl))};
          const F2 g = {make_float2(gpre[pa], has2 ? gpre[pb] : 0.f)};
          ray_adj(sv, sv.an, sv.ant, x, y, g, acc);
        }
      }
#else
      {
        for (int p = p0 + threadIdx.x; p < p1; p += stride) {
          const int i = p / W, j = p - i * W;
          const float g = gpre[p];
          for (int a = 0; a < k; ++a) {
            const float y = grid_coord(2 * (i * k + a) + ss.ny0, ss.hh, ss.hl);
            for (int c = 0; c < k; ++c) {
              const float x = grid_coord(2 * (j * k + c) + ss.nx0, ss.hh, ss.hl);
              ray_adj(sv, sv.an, sv.ant, x, y, g, acc);
            }
          }
        }
      }
#endif
    }
    // pairwise FP32 sums within the warp (GB300's FP64 pipe is narrow), FP64 across warps
#pragma unroll
    for (int a = 0; a < NACC; ++a) {
      float v = lane_sum(acc[a]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][a] = double(v);
    }
    __syncthreads();
    if (threadIdx.x < NACC) {
      double v = 0.0;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
      ss.partial[(size_t(b) * ss.ntiles + tile) * NACC + threadIdx.x] = v;
    }
    __syncthreads();
  }
}

// -------------------------------------------------------------- k_conv ----

// out(i, j) = sum_{a,b} ker[a K + b] in[(i + a) Wp + j + b] for the R rows
// i = i0 .. i0 + R - 1 of column j. The kernel column sits in registers and
// every input value is read once per kernel column.
template <int K, int R>
__device__ __forceinline__ void corr_strip(const float* in, int Wp, const float* ker, int i0, int j, float* acc) {
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.f;
  const float* base = in + i0 * Wp + j;
#pragma unroll 1
  for (int b = 0; b < K; ++b) {
    float kc[K];
#pragma unroll
    for (int a = 0; a < K; ++a) kc[a] = ker[a * K + b];
    const float* col = base + b;
#pragma unroll
    for (int ii = 0; ii < R + K - 1; ++ii) {
      const float v = col[ii * Wp];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int a = ii - r;
        if (a >= 0 && a < K) acc[r] = fmaf(kc[a], v, acc[r]);
      }
    }
  }
}

template <int R>
__device__ __forceinline__ void corr_strip_any(const float* in, int Wp, const float* ker, int K, int i0, int j,
                                               float* acc) {
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.f;
  const float* base = in + i0 * Wp + j;
  for (int b = 0; b < K; ++b) {
    const float* col = base + b;
    for (int ii = 0; ii < R + K - 1; ++ii) {
      const float v = col[ii * Wp];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int a = ii - r;
        if (a >= 0 && a < K) acc[r] = fmaf(ker[a * K + b], v, acc[r]);
      }
    }
  }
}

// Columns per strip row of work units: a multiple of 32, so that a warp's
// lanes read 32 consecutive shared-memory words of one image row.
__device__ __forceinline__ int conv_row_units(int W) { return (W + 31) & ~31; }

// Row pitch (floats) of the row-strip convolution: room for 16-column strips
// plus the K - 1 halo, a multiple of 4 with an odd number of float4 per row.
__host__ __device__ inline int rowconv_pitch(int W, int K) {
  int P = ((W + 15) / 16) * 16 + K - 1;
  P = (P + 3) & ~3;
  if (((P >> 2) & 1) == 0) P += 4;
  return P;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One vector. Shared memory: PSF flipped (convolution) and as given
// (correlation), the zero-padded binned image and, when it fits
// (s.conv_two_buf), a second zero-padded buffer for the pixel adjoint;
// otherwise the adjoint goes through this vector's global work slot.
// K > 0: compile-time PSF side; K == 0: any odd side (s.K).
template <int K, int R>
__device__ void conv_vector(const Seg& s, int b, int mode, float* smem, double* red2) {
  const int Kk = K > 0 ? K : s.K;
  const int H = s.H, W = s.W, HW = H * W;
  const int nstrip = (H + R - 1) / R;
  const int Hp = nstrip * R + Kk - 1, Wp = W + Kk - 1;
  const int c = (Kk - 1) / 2;
  const int K2 = (Kk * Kk + 3) & ~3;
  float* kerF = smem;
  float* kerU = smem + K2;
  float* img = smem + 2 * K2;
  float* img2 = img + Hp * Wp;
  float* work = s.work + size_t(b) * HW;
  const bool want_sim = (mode == MODE_SIM);
  const bool corr_only = (mode == MODE_CORR);   // the work slot holds d log L / d M already
  const bool want_grad = (mode == MODE_GRAD) || corr_only;
  const bool two = (mode == MODE_GRAD) && s.conv_two_buf;

  for (int i = threadIdx.x; i < Kk * Kk; i += blockDim.x) {
    kerF[i] = s.psf[Kk * Kk - 1 - i];
    kerU[i] = s.psf[i];
  }
  const int nz = (two ? 2 : 1) * Hp * Wp;
  for (int i = threadIdx.x; i < nz; i += blockDim.x) img[i] = 0.f;
  __syncthreads();
#pragma unroll 4
  for (int p = threadIdx.x; p < HW; p += blockDim.x) {
    const int i = p / W, j = p - i * W;
    img[(i + c) * Wp + j + c] = work[p];
  }
  __syncthreads();

  float ll = 0.f, c2 = 0.f;
  const int Wr = conv_row_units(W);
  const int units = nstrip * Wr;
  float acc[R];
  if (!corr_only) {
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    const int strip = u / Wr, j = u - strip * Wr;
    if (j >= W) continue;
    const int i0 = strip * R;
    if (K > 0) corr_strip<(K > 0 ? K : 1), R>(img, Wp, kerF, i0, j, acc);
    else corr_strip_any<R>(img, Wp, kerF, Kk, i0, j, acc);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = i0 + r;
      if (i < H) {
        const int p = i * W + j;
        const float M = acc[r];
        if (want_sim) {
          s.sim[size_t(b) * HW + p] = M;
        } else {
          const float v = fmaf(M, s.inv_gain, s.sigma2[p]);
          const float res = s.image[p] - M;
          const float iv = 1.0f / v;
          const float t2 = res * res * iv;
          c2 += t2;
          ll += t2 + logf(6.28318530717958648f * v);
          if (want_grad) {
            // d log L / d M = res/v + (res^2/v^2 - 1/v) / (2 G t_exp)
            const float gm = fmaf(0.5f * s.inv_gain, fmaf(t2, iv, -iv), res * iv);
            if (two) img2[(i + c) * Wp + j + c] = gm;
            else work[p] = gm;
          }
        }
      }
    }
  }
  if (!want_sim) {
    // FP32 within a thread (a few tens of pixels) and a warp (pairwise), FP64 across warps
    ll = warp_sum_f(ll);
    c2 = warp_sum_f(c2);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
      red2[2 * warp] = double(ll);
      red2[2 * warp + 1] = double(c2);
    }
  }
  __syncthreads();
  if (!want_sim && threadIdx.x == 0) {
    double L = 0.0, C = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      L += red2[2 * w];
      C += red2[2 * w + 1];
    }
    if (s.loglik) s.loglik[b] = -0.5 * L;
    if (s.chi2) s.chi2[b] = C;
  }
  if (!want_grad) return;
  }   // !corr_only

  // adjoint: gpre = (PSF correlated with dlogL/dM) / k^2
  float* gsrc = img2;
  if (corr_only) {
    gsrc = img;   // loaded from the work slot above
  } else if (!two) {
#pragma unroll 4
    for (int p = threadIdx.x; p < HW; p += blockDim.x) {
      const int i = p / W, j = p - i * W;
      img[(i + c) * Wp + j + c] = work[p];
    }
    __syncthreads();
    gsrc = img;
  }
  const float inv_k2 = 1.0f / float(s.k * s.k);
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    const int strip = u / Wr, j = u - strip * Wr;
    if (j >= W) continue;
    const int i0 = strip * R;
    if (K > 0) corr_strip<(K > 0 ? K : 1), R>(gsrc, Wp, kerU, i0, j, acc);
    else corr_strip_any<R>(gsrc, Wp, kerU, Kk, i0, j, acc);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = i0 + r;
      if (i < H) work[i * W + j] = acc[r] * inv_k2;
    }
  }
}

// Likelihood terms of pixel p with model value M (Eq. for log L with the
// model-dependent variance): adds chi^2 and chi^2 + log(2 pi v) to c2 and ll
// and returns d log L / d M. Explicit roundings: the log-L-only and gradient
// calls give identical sums. 1/v and log(2 pi v) by the hardware
// approximations (relative error ~1e-7, far below the likelihood's FP32
// summation error).
__device__ __forceinline__ float pixel_terms(const Seg& s, int p, float M, float& ll, float& c2) {
  const float v = fmaf(M, s.inv_gain, s.sigma2[p]);
  const float res = __fsub_rn(s.image[p], M);
  const float iv = rcp(v);
  const float t2 = __fmul_rn(__fmul_rn(res, res), iv);
  c2 = __fadd_rn(c2, t2);
  ll = __fadd_rn(ll, __fadd_rn(t2, __fmul_rn(0.69314718055994531f, lg2(__fmul_rn(6.28318530717958648f, v)))));
  // d log L / d M = res/v + (res^2/v^2 - 1/v) / (2 G t_exp)
  return fmaf(0.5f * s.inv_gain, fmaf(t2, iv, -iv), res * iv);
}

// ---- row-strip convolution for the compile-time PSF sides (11, 21) ----
//
// Each thread computes S = 16 consecutive outputs of one image row; the lanes
// of a warp take consecutive rows. Per kernel row a thread loads the input
// span (S + K - 1 values) and the kernel row as float4 and does S*K FMAs from
// registers. The row pitch P (floats) is a multiple of 4 with an odd number
// of float4 per row, so the 8 lanes of each 128-bit shared-memory phase hit
// 8 distinct bank groups.

// out[r] = sum_{a,b} ker[a][b] in[(i + a) P + j0 + r + b], r < 16; ker rows of KP floats.
template <int K>
__device__ __forceinline__ void corr_row(const float* __restrict__ in, int P, const float* __restrict__ ker, int i,
                                         int j0, float (&acc)[16]) {
  constexpr int S = 16, KP = (K + 3) & ~3, NIN = (S + K - 1 + 3) & ~3;
#pragma unroll
  for (int r = 0; r < S; ++r) acc[r] = 0.f;
  const float* row = in + i * P + j0;
#pragma unroll 1
  for (int a = 0; a < K; ++a) {
    float x[NIN];
    const float4* r4 = reinterpret_cast<const float4*>(row + a * P);
#pragma unroll
    for (int q = 0; q < NIN / 4; ++q) {
      const float4 t = r4[q];
      x[4 * q] = t.x;
      x[4 * q + 1] = t.y;
      x[4 * q + 2] = t.z;
      x[4 * q + 3] = t.w;
    }
    float kr[KP];
    const float4* k4 = reinterpret_cast<const float4*>(ker + a * KP);
#pragma unroll
    for (int q = 0; q < KP / 4; ++q) {
      const float4 t = k4[q];
      kr[4 * q] = t.x;
      kr[4 * q + 1] = t.y;
      kr[4 * q + 2] = t.z;
      kr[4 * q + 3] = t.w;
    }
#pragma unroll
    for (int b = 0; b < K; ++b) {
#pragma unroll
      for (int r = 0; r < S; ++r) acc[r] = fmaf(kr[b], x[r + b], acc[r]);
    }
  }
}

// 4-byte asynchronous global -> shared copy (completes at cp_async_wait_all).
__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gsrc) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// The binned image (the vector's work slot) into the interior of the
// zero-padded buffer img ([H + K - 1][P], halo (K - 1)/2), by asynchronous
// copies while the halo is zeroed; rows across warps, columns across lanes.
// The caller synchronises the block after.
template <int K>
__device__ __forceinline__ void load_padded(const Seg& s, float* img, int P, const float* work) {
  constexpr int c = (K - 1) / 2;
  const int H = s.H, W = s.W;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < H; i += nw)
    for (int j = lane; j < W; j += 32) cp_async4(&img[(i + c) * P + j + c], &work[i * W + j]);
  for (int i = threadIdx.x; i < c * P; i += blockDim.x) {
    img[i] = 0.f;                       // top halo rows
    img[(H + c) * P + i] = 0.f;         // bottom halo rows
  }
  const int side = P - W;               // left halo c columns + right halo and pitch padding
  for (int t = threadIdx.x; t < H * side; t += blockDim.x) {
    const int i = t / side, q = t - i * side;
    img[(i + c) * P + (q < c ? q : W + q)] = 0.f;
  }
  cp_async_wait_all();
}

// log L and chi^2 of the block's vector from the threads' partial sums (FP32
// within a warp, pairwise; FP64 across warps in warp order), and a block
// barrier: every thread calls it.
__device__ __forceinline__ void block_loglik(const Seg& s, int b, float ll, float c2, double* red2) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  ll = warp_sum_f(ll);
  c2 = warp_sum_f(c2);
  if (lane == 0) {
    red2[2 * wid] = double(ll);
    red2[2 * wid + 1] = double(c2);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double L = 0.0, C = 0.0;
    for (int w = 0; w < nw; ++w) {
      L += red2[2 * w];
      C += red2[2 * w + 1];
    }
    if (s.loglik) s.loglik[b] = -0.5 * L;
    if (s.chi2) s.chi2[b] = C;
  }
}

// Pixel phase after the model pass (coalesced: rows across warps, columns
// across lanes): the model value of pixel (i, j) from stage (pitch P) if two,
// else from the work slot. With want_sim it goes to s.sim; otherwise the
// likelihood terms are summed (FP32 within a thread and a warp, pairwise;
// FP64 across warps: the block size sets the summation order, the last bits
// of log L) into s.loglik / s.chi2, and with want_grad d log L / d M goes
// into img's interior (halo c). Returns whether a correlation pass follows.
__device__ bool pixel_phase(const Seg& s, int b, bool want_sim, bool want_grad, const float* stage, int P, float* img,
                            int c, bool two, double* red2) {
  const int H = s.H, W = s.W, HW = H * W;
  const float* work = s.work + size_t(b) * HW;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float ll = 0.f, c2 = 0.f;
  for (int i = wid; i < H; i += nw)
#pragma unroll 2
  for (int j = lane; j < W; j += 32) {
    const int p = i * W + j;
    const float M = two ? stage[i * P + j] : work[p];
    if (want_sim) {
      s.sim[size_t(b) * HW + p] = M;
      continue;
    }
    const float gm = pixel_terms(s, p, M, ll, c2);
    if (want_grad) img[(i + c) * P + j + c] = gm;
  }
  if (!want_sim)
    block_loglik(s, b, ll, c2, red2);
  else
    __syncthreads();
  return want_grad;
}

// One vector, PSF side K known at compile time. Shared memory: both PSF
// orientations ([K][KP], zero padded), the zero-padded input buffer
// [H + K - 1][P] and, when s.conv_two_buf, an unpadded staging buffer [H][P]
// for the model values and the correlation output (else they go through the
// vector's global work slot). After the first pass the input buffer's
// interior is overwritten with d log L / d M (its zero halo is reused).
template <int K>
__device__ void conv_vector_rows(const Seg& s, int b, int mode, float* smem, double* red2) {
  constexpr int S = 16, KP = (K + 3) & ~3, c = (K - 1) / 2;
  const int H = s.H, W = s.W, HW = H * W;
  const int P = rowconv_pitch(W, K);
  const int Hp = H + K - 1;
  float* kerF = smem;
  float* kerU = smem + K * KP;
  float* img = smem + 2 * K * KP;
  float* stage = img + Hp * P;
  float* work = s.work + size_t(b) * HW;
  const bool want_sim = (mode == MODE_SIM);
  const bool corr_only = (mode == MODE_CORR);   // the work slot holds d log L / d M already
  const bool want_grad = (mode == MODE_GRAD) || corr_only;
  const bool two = s.conv_two_buf != 0;

  for (int i = threadIdx.x; i < K * KP; i += blockDim.x) {
    const int a = i / KP, bb = i - a * KP;
    kerF[i] = bb < K ? s.psf[(K - 1 - a) * K + (K - 1 - bb)] : 0.f;
    kerU[i] = bb < K ? s.psf[a * K + bb] : 0.f;
  }
  // pixel loops: rows across warps, columns across lanes (coalesced, no division)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  load_padded<K>(s, img, P, work);
  __syncthreads();

  const int nstrip = (W + S - 1) / S;
  const int units = nstrip * H;
  float acc[S];
  if (!corr_only) {
  // pass 1: model image M (convolution with the flipped PSF)
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    const int strip = u / H, i = u - strip * H, j0 = strip * S;
    corr_row<K>(img, P, kerF, i, j0, acc);
    if (two) {
      float4* o4 = reinterpret_cast<float4*>(stage + i * P + j0);
#pragma unroll
      for (int q = 0; q < S / 4; ++q) o4[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    } else {
#pragma unroll
      for (int r = 0; r < S; ++r)
        if (j0 + r < W) work[i * W + j0 + r] = acc[r];
    }
  }
  __syncthreads();

  if (!pixel_phase(s, b, want_sim, want_grad, stage, P, img, c, two, red2)) return;
  }   // !corr_only

  // pass 2: subpixel adjoint = (PSF correlated with d log L / d M) / k^2
  const float inv_k2 = 1.0f / float(s.k * s.k);
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    const int strip = u / H, i = u - strip * H, j0 = strip * S;
    corr_row<K>(img, P, kerU, i, j0, acc);
    if (two) {
      float4* o4 = reinterpret_cast<float4*>(stage + i * P + j0);
#pragma unroll
      for (int q = 0; q < S / 4; ++q)
        o4[q] = make_float4(acc[4 * q] * inv_k2, acc[4 * q + 1] * inv_k2, acc[4 * q + 2] * inv_k2,
                            acc[4 * q + 3] * inv_k2);
    } else {
#pragma unroll
      for (int r = 0; r < S; ++r)
        if (j0 + r < W) work[i * W + j0 + r] = acc[r] * inv_k2;
    }
  }
  if (two) {
    __syncthreads();
    for (int i = wid; i < H; i += nw)
      for (int j = lane; j < W; j += 32) work[i * W + j] = stage[i * P + j];
  }
}

// ---- separable PSFs: the convolution as 1-D passes ----
//
// A PSF whose singular values beyond the first R are negligible (psf_rank,
// from gl_system_create: their root sum of squares is at most 2^-24 of the
// PSF's Frobenius norm, the rounding its FP32 entries already carry) is
// P = sum_r u_r v_r^T (u_r carries the singular value). A pass over the
// image is then R horizontal K-tap passes (v_r, into R row buffers) and, per
// output, the sum over r of K-tap vertical passes (u_r): 2 K R multiply-adds
// per pixel instead of K^2 (a sampled Gaussian PSF has R = 1: 22 instead of
// 121 at K = 11). flip: the flipped PSF (the model's convolution), else the
// PSF (the adjoint's correlation).
constexpr int SEP_RV = 8;   // output rows per unit of the vertical pass

// Shared memory of the separable form: the factors [R][2][K] (u_r, v_r), the
// u_r taps again as duplicated pairs [R][K] (for packed FMAs), the
// zero-padded input [Ht][P] and R row buffers [Ht][P]; Ht = H rounded up to
// whole vertical units, plus K - 1 halo rows, so that no vertical unit reads
// past a buffer. The same formula sizes the launch (conv_sep_smem_bytes).
struct SepLayout {
  int P, Ht, nvs;
  float* fac;
  float2* tapu;
  float* img;
  float* tmp;
};

__host__ __device__ inline int sep_rows(int H, int K) { return (H + SEP_RV - 1) / SEP_RV * SEP_RV + K - 1; }

// rows: the output rows a block covers (the image, or a band of it)
__device__ __forceinline__ SepLayout sep_layout(const Seg& s, float* smem, int rows) {
  SepLayout L;
  L.P = rowconv_pitch(s.W, s.K);
  L.Ht = sep_rows(rows, s.K);
  L.nvs = (rows + SEP_RV - 1) / SEP_RV;
  const int nf = (2 * s.psf_rank * s.K + 3) & ~3;
  L.fac = smem;
  L.tapu = reinterpret_cast<float2*>(smem + nf);
  L.img = smem + 2 * nf;
  L.tmp = L.img + L.Ht * L.P;
  return L;
}

// The factors into shared memory and the input buffer's halo (everything
// outside rows c .. c + H - 1, columns c .. c + W - 1) zeroed; rows across
// warps, columns across lanes. The caller synchronises the block before
// the factors are read.
template <int K>
__device__ __forceinline__ void sep_prepare(const Seg& s, const SepLayout& L) {
  constexpr int c = (K - 1) / 2;
  const int R = s.psf_rank;
  for (int i = threadIdx.x; i < 2 * R * K; i += blockDim.x) L.fac[i] = s.psf_sep[i];
  for (int i = threadIdx.x; i < R * K; i += blockDim.x) {
    const float u = s.psf_sep[(i / K) * 2 * K + i % K];
    L.tapu[i] = make_float2(u, u);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < L.Ht; i += nw) {
    const bool inner = i >= c && i < c + s.H;
    for (int q = lane; q < L.P; q += 32)
      if (!inner || q < c || q >= c + s.W) L.img[i * L.P + q] = 0.f;
  }
}

// The binned image (the vector's work slot) into the input's interior by
// asynchronous copies, issued only: the caller waits for them
// (cp_async_wait_all) and synchronises the block.
template <int K>
__device__ __forceinline__ void sep_load_issue(const Seg& s, const SepLayout& L, const float* work) {
  constexpr int c = (K - 1) / 2;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < s.H; i += nw)
    for (int j = lane; j < s.W; j += 32) cp_async4(&L.img[(i + c) * L.P + j + c], &work[i * s.W + j]);
}

// Horizontal passes: row buffer r, row i, columns j0 .. j0 + 15, for the Ht
// rows. A warp takes 32 consecutive rows of one strip (float4 loads of rows
// an odd number of 16-byte words apart are conflict-free); each unit loads
// its input span once for the R terms. FLIP: the flipped factor (the model's
// convolution); RC: the rank when known at compile time (1), else 0.
template <int K, bool FLIP, int RC>
__device__ __forceinline__ void sep_hpass(const float* __restrict__ in, const SepLayout& L, int W, int Rrt) {
  constexpr int S = 16, NIN = (S + K - 1 + 3) & ~3;
  const int R = RC > 0 ? RC : Rrt;
  const int P = L.P, Ht = L.Ht, nstrip = (W + S - 1) / S, rg = (Ht + 31) >> 5, tasks = nstrip * rg;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int strip = wid / rg, g = wid - strip * rg;   // task w = strip * rg + g, stepped without division
  for (int w = wid; w < tasks; w += nw) {
    const int i = g * 32 + lane, j0 = strip * S;
    g += nw;
    while (g >= rg) {
      g -= rg;
      ++strip;
    }
    if (i >= Ht) continue;
    float x[NIN];
    const float4* r4 = reinterpret_cast<const float4*>(in + i * P + j0);
#pragma unroll
    for (int q = 0; q < NIN / 4; ++q) {
      const float4 v = r4[q];
      x[4 * q] = v.x;
      x[4 * q + 1] = v.y;
      x[4 * q + 2] = v.z;
      x[4 * q + 3] = v.w;
    }
    for (int r = 0; r < R; ++r) {
      const float* v = L.fac + (2 * r + 1) * K;
      float acc[S];
#pragma unroll
      for (int o = 0; o < S; ++o) {
        float a = 0.f;
#pragma unroll
        for (int q = 0; q < K; ++q) a = fmaf(v[FLIP ? K - 1 - q : q], x[o + q], a);
        acc[o] = a;
      }
      float4* t4 = reinterpret_cast<float4*>(L.tmp + size_t(r) * Ht * P + i * P + j0);
#pragma unroll
      for (int q = 0; q < S / 4; ++q) t4[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
  }
}

// Vertical passes of one unit: rows i0 .. i0 + 7 of columns j, j + 1 (j
// even) in packed pairs, summed over the R terms (per lane the FMAs of the
// scalar form, in the same order).
template <int K, bool FLIP, int RC>
__device__ __forceinline__ void sep_vunit(const SepLayout& L, int Rrt, int i0, int j, float2 (&m)[SEP_RV]) {
  constexpr int NV = SEP_RV + K - 1;
  const int R = RC > 0 ? RC : Rrt;
#pragma unroll
  for (int o = 0; o < SEP_RV; ++o) m[o] = make_float2(0.f, 0.f);
  for (int r = 0; r < R; ++r) {
    const float2* tap = L.tapu + r * K;
    const float* col = L.tmp + size_t(r) * L.Ht * L.P + i0 * L.P + j;
    float2 x[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) x[q] = *reinterpret_cast<const float2*>(col + q * L.P);
#pragma unroll
    for (int o = 0; o < SEP_RV; ++o) {
      float2 a = m[o];
#pragma unroll
      for (int q = 0; q < K; ++q) a = __ffma2_rn(tap[FLIP ? K - 1 - q : q], x[o + q], a);
      m[o] = a;
    }
  }
}

// Calls f(i0, j) for every vertical unit of nvs strips of 8 rows and Wp2
// column pairs. Where a block's threads cover at least one strip's pairs,
// thread t keeps column pair t % Wp2 and steps through the strips
// (one division per call); else the units are spread over all threads.
template <class F>
__device__ __forceinline__ void for_vunits(int nvs, int Wp2, F&& f) {
  const int spr = blockDim.x / Wp2;   // strips per round
  if (spr > 0) {
    const int s0 = threadIdx.x / Wp2, jp = threadIdx.x - s0 * Wp2;
    if (s0 < spr)
      for (int strip = s0; strip < nvs; strip += spr) f(strip * SEP_RV, 2 * jp);
  } else {
    for (int u = threadIdx.x; u < nvs * Wp2; u += blockDim.x) {
      const int strip = u / Wp2;
      f(strip * SEP_RV, 2 * (u - strip * Wp2));
    }
  }
}

// One vector with a separable PSF (s.conv_sep), its halo and factors in
// place when prepared (a single-system kernel prepares once per block), else
// set up here. The model pass's vertical step computes the likelihood terms
// of its outputs at once and writes d log L / d M over the input's interior
// (the horizontal step has read it); the correlation's vertical step writes
// the subpixel adjoint to the vector's work slot. Every pixel's model value,
// likelihood terms and adjoint are fixed by the layout, not the block size;
// log L is summed in a block-size-dependent order. MODE_T: the mode when
// known at compile time, else -1 (mode_rt); RC as for sep_hpass. PF (with
// MODE_T the gradient mode): this vector's image copies were issued by the
// caller, and the copies of vector next_b (if >= 0) are issued once the
// correlation's horizontal pass has read the input, so that they run during
// the vertical pass.
template <int K, int MODE_T, int RC, bool PF = false>
__device__ void conv_vector_sep(const Seg& s, int b, int mode_rt, float* smem, double* red2, bool prepared,
                                int next_b = -1) {
  static_assert(!PF || MODE_T == MODE_GRAD, "prefetch only in the gradient pass");
  constexpr int c = (K - 1) / 2;
  const int mode = MODE_T >= 0 ? MODE_T : mode_rt;
  const int H = s.H, W = s.W, HW = H * W, R = RC > 0 ? RC : s.psf_rank;
  const SepLayout L = sep_layout(s, smem, H);
  float* work = s.work + size_t(b) * HW;
  const bool want_sim = (mode == MODE_SIM);
  const bool corr_only = (mode == MODE_CORR);   // the work slot holds d log L / d M already
  const bool want_grad = (mode == MODE_GRAD) || corr_only;
  const int Wp2 = (W + 1) >> 1;
  if (!prepared) sep_prepare<K>(s, L);
  if (!PF) sep_load_issue<K>(s, L, work);
  cp_async_wait_all();
  __syncthreads();
  if (!corr_only) {
    sep_hpass<K, true, RC>(L.img, L, W, R);
    __syncthreads();
    float ll = 0.f, c2 = 0.f;
    for_vunits(L.nvs, Wp2, [&](int i0, int j) {
      const bool two = j + 1 < W;
      float2 m[SEP_RV];
      sep_vunit<K, true, RC>(L, R, i0, j, m);
#pragma unroll
      for (int o = 0; o < SEP_RV; ++o) {
        const int i = i0 + o;
        if (i >= H) break;
        const int p = i * W + j;
        if (want_sim) {
          s.sim[size_t(b) * HW + p] = m[o].x;
          if (two) s.sim[size_t(b) * HW + p + 1] = m[o].y;
          continue;
        }
        const float g0 = pixel_terms(s, p, m[o].x, ll, c2);
        if (want_grad) L.img[(i + c) * L.P + j + c] = g0;
        if (two) {
          const float g1 = pixel_terms(s, p + 1, m[o].y, ll, c2);
          if (want_grad) L.img[(i + c) * L.P + j + 1 + c] = g1;
        }
      }
    });
    if (want_sim) return;
    block_loglik(s, b, ll, c2, red2);   // also the barrier before the correlation reads img
    if (!want_grad) return;
  }
  sep_hpass<K, false, RC>(L.img, L, W, R);
  __syncthreads();
  if (PF && next_b >= 0) sep_load_issue<K>(s, L, s.work + size_t(next_b) * HW);
  const float inv_k2 = 1.0f / float(s.k * s.k);
  for_vunits(L.nvs, Wp2, [&](int i0, int j) {
    float2 m[SEP_RV];
    sep_vunit<K, false, RC>(L, R, i0, j, m);
#pragma unroll
    for (int o = 0; o < SEP_RV; ++o) {
      const int i = i0 + o;
      if (i >= H) break;
      work[i * W + j] = m[o].x * inv_k2;
      if (j + 1 < W) work[i * W + j + 1] = m[o].y * inv_k2;
    }
  });
}

template <int K, int R, int NT, int MINB, class Src>
__global__ void __launch_bounds__(NT, MINB) k_conv(const __grid_constant__ Src src, int mode) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  __shared__ double red2[2 * (NT / 32)];
  __shared__ Seg ss;
  const PdlScope pdl;
  for (int item = blockIdx.x; item < src.nconv(); item += gridDim.x) {
    int b;
    const Seg* segp = src.conv_seg(item, b);
    block_copy(&ss, segp);
    __syncthreads();
    if constexpr (K > 0) {
      // a single-system call takes k_conv_sep for a separable PSF; a table
      // may mix both kinds of segment
      if (!std::is_same<Src, OneSeg>::value && ss.conv_sep)
        conv_vector_sep<K, -1, 0>(ss, b, mode, smem, red2, false);
      else
        conv_vector_rows<K>(ss, b, mode, smem, red2);
    } else {
      conv_vector<K, R>(ss, b, mode, smem, red2);
    }
    __syncthreads();
  }
}

// The separable convolution of a single-system call (its own kernel, so that
// the 2-D form's register budget does not bound it).
template <int K, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_conv_sep(const __grid_constant__ OneSeg src, int mode) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  __shared__ double red2[2 * (NT / 32)];
  const PdlScope pdl;
  // the factors and the zero halo stay in place for all of the block's
  // vectors; each vector's steps end with the vertical pass, which reads only
  // the row buffers, and the next vector's horizontal pass comes after the
  // barrier that follows its image load
  sep_prepare<K>(src.s, sep_layout(src.s, smem, src.s.H));
  // the gradient call of a rank-1 PSF (a sampled Gaussian) with its mode and
  // rank known at compile time; any other call with both read at run time
  if (mode == MODE_GRAD && src.s.psf_rank == 1) {
    // each vector's image copies run during the previous vector's last pass
    const int n = src.nconv();
    if (int(blockIdx.x) < n)
      sep_load_issue<K>(src.s, sep_layout(src.s, smem, src.s.H), src.s.work + size_t(blockIdx.x) * src.s.H * src.s.W);
    for (int item = blockIdx.x; item < n; item += gridDim.x) {
      const int next = item + int(gridDim.x);
      conv_vector_sep<K, MODE_GRAD, 1, true>(src.s, item, mode, smem, red2, true, next < n ? next : -1);
    }
  } else {
    for (int item = blockIdx.x; item < src.nconv(); item += gridDim.x)
      conv_vector_sep<K, -1, 0>(src.s, item, mode, smem, red2, true);
  }
}

// ---- small batches: one vector's convolution over a cluster of row bands ----
//
// Below half as many vectors as SMs, one block per vector leaves most SMs
// idle. Here a thread-block cluster of nb blocks shares a vector: block r
// convolves output rows [r rows, (r + 1) rows) from its band and the K - 1
// halo rows of the binned image (global memory), evaluates the likelihood
// terms of its rows and keeps their d log L / d M in shared memory. After a
// cluster barrier each block copies the d log L / d M halo rows it needs out
// of its neighbours' shared memory (distributed shared memory) and block 0
// adds the bands' log L and chi^2 in rank order; after a second barrier (no
// block reads another's shared memory beyond it) each block correlates its
// rows with the PSF. Per pixel the arithmetic is that of conv_vector_rows,
// so gradients are the same bits; log L is summed in a band-dependent order.
constexpr int BAND_THREADS = 256;

__host__ __device__ inline size_t conv_band_smem_bytes(int W, int K, int rows) {
  const size_t KP = size_t((K + 3) & ~3), P = size_t(rowconv_pitch(W, K));
  return (2 * size_t(K) * KP + (size_t(rows) + K - 1) * P + size_t(rows) * P) * sizeof(float);
}

template <int K>
__global__ void __launch_bounds__(BAND_THREADS) k_conv_bands(const __grid_constant__ OneSeg src, int mode, int rows) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  __shared__ double red2[2 * (BAND_THREADS / 32)];
  __shared__ double band_sum[2];
  const PdlScope pdl;
  constexpr int S = 16, KP = (K + 3) & ~3, c = (K - 1) / 2;
  const Seg& s = src.s;
  const int nb = int(cluster.num_blocks()), rank = int(cluster.block_rank());
  const int b = blockIdx.x / nb;
  const int H = s.H, W = s.W, HW = H * W;
  const int P = rowconv_pitch(W, K);
  const int r0 = min(H, rank * rows), nr = min(H, r0 + rows) - r0;   // nr may be 0
  const int Hb = rows + K - 1;
  float* kerF = smem;
  float* kerU = smem + K * KP;
  float* img = smem + 2 * K * KP;   // [Hb][P], local row li holds image row r0 - c + li
  float* stage = img + Hb * P;      // [rows][P]
  float* work = s.work + size_t(b) * HW;
  const bool want_sim = (mode == MODE_SIM);
  const bool want_grad = (mode == MODE_GRAD);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;

  for (int i = threadIdx.x; i < K * KP; i += blockDim.x) {
    const int a = i / KP, bb = i - a * KP;
    kerF[i] = bb < K ? s.psf[(K - 1 - a) * K + (K - 1 - bb)] : 0.f;
    kerU[i] = bb < K ? s.psf[a * K + bb] : 0.f;
  }
  for (int li = wid; li < Hb; li += nw) {
    const int g = r0 - c + li;
    float* row = img + li * P;
    if (g >= 0 && g < H) {
      for (int j = lane; j < W; j += 32) cp_async4(&row[j + c], &work[g * W + j]);
      for (int q = lane; q < P - W; q += 32) row[q < c ? q : W + q] = 0.f;
    } else {
      for (int j = lane; j < P; j += 32) row[j] = 0.f;
    }
  }
  cp_async_wait_all();
  __syncthreads();

  // pass 1: M of this band's rows
  const int nstrip = (W + S - 1) / S;
  const int units = nstrip * nr;
  float acc[S];
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    const int strip = u / nr, li = u - strip * nr, j0 = strip * S;
    corr_row<K>(img, P, kerF, li, j0, acc);
    float4* o4 = reinterpret_cast<float4*>(stage + li * P + j0);
#pragma unroll
    for (int q = 0; q < S / 4; ++q) o4[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
  }
  __syncthreads();

  // pixel phase of the band: likelihood terms, d log L / d M into img's interior
  float ll = 0.f, c2 = 0.f;
  for (int li = wid; li < nr; li += nw)
#pragma unroll 2
    for (int j = lane; j < W; j += 32) {
      const int p = (r0 + li) * W + j;
      const float M = stage[li * P + j];
      if (want_sim) {
        s.sim[size_t(b) * HW + p] = M;
        continue;
      }
      const float gm = pixel_terms(s, p, M, ll, c2);
      if (want_grad) img[(li + c) * P + j + c] = gm;
    }
  ll = warp_sum_f(ll);
  c2 = warp_sum_f(c2);
  if (lane == 0) {
    red2[2 * wid] = double(ll);
    red2[2 * wid + 1] = double(c2);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double L = 0.0, C = 0.0;
    for (int w = 0; w < nw; ++w) {
      L += red2[2 * w];
      C += red2[2 * w + 1];
    }
    band_sum[0] = L;
    band_sum[1] = C;
  }
  cluster.sync();   // every band's d log L / d M and sums are in its shared memory
  if (!want_sim && rank == 0 && threadIdx.x == 0) {
    double L = 0.0, C = 0.0;
    for (int r = 0; r < nb; ++r) {
      const double* bs = cluster.map_shared_rank(band_sum, r);
      L += bs[0];
      C += bs[1];
    }
    if (s.loglik) s.loglik[b] = -0.5 * L;
    if (s.chi2) s.chi2[b] = C;
  }
  if (want_grad) {
    // the halo rows of d log L / d M from the bands that own them
    for (int li = wid; li < Hb; li += nw) {
      if (li >= c && li < c + nr) continue;
      const int g = r0 - c + li;
      if (g < 0 || g >= H) continue;   // stays zero
      const int owner = g / rows;
      const float* oimg = cluster.map_shared_rank(img, owner);
      const float* orow = oimg + (g - owner * rows + c) * P + c;
      for (int j = lane; j < W; j += 32) img[li * P + j + c] = orow[j];
    }
  }
  cluster.sync();   // no block reads another's shared memory after this barrier
  if (!want_grad) return;

  // pass 2: subpixel adjoint of the band's rows = (PSF correlated with d log L / d M) / k^2
  const float inv_k2 = 1.0f / float(s.k * s.k);
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    const int strip = u / nr, li = u - strip * nr, j0 = strip * S;
    corr_row<K>(img, P, kerU, li, j0, acc);
    float4* o4 = reinterpret_cast<float4*>(stage + li * P + j0);
#pragma unroll
    for (int q = 0; q < S / 4; ++q)
      o4[q] = make_float4(acc[4 * q] * inv_k2, acc[4 * q + 1] * inv_k2, acc[4 * q + 2] * inv_k2,
                          acc[4 * q + 3] * inv_k2);
  }
  __syncthreads();
  for (int li = wid; li < nr; li += nw)
    for (int j = lane; j < W; j += 32) work[(r0 + li) * W + j] = stage[li * P + j];
}

// ---- separable PSFs over a cluster of row bands ----
//
// The separable form for a vector whose whole-image buffers do not fit one
// block's shared memory (200 x 200, K = 21), and for small batches (below
// half as many vectors as SMs). A cluster of nb blocks shares the vector as
// in k_conv_bands: block r holds its band's input rows with the K - 1 halo
// rows (from the work slot), runs the horizontal and the fused vertical and
// likelihood passes for its rows, and keeps d log L / d M of its rows over
// its input's interior. After a cluster barrier it copies its halo rows of
// d log L / d M from the blocks that own them (distributed shared memory)
// and block 0 adds the bands' log L and chi^2 in rank order; after a second
// barrier (no remote reads beyond it) each block correlates its rows. Per
// pixel the arithmetic is that of conv_vector_sep (same factors, taps and
// order), so the gradient bits do not depend on the banding. With
// MODE_CORR the work slot already holds d log L / d M: each block loads its
// rows with their halo and the blocks meet at a barrier before any of them
// writes the work slot.
__host__ __device__ inline size_t conv_sep_band_smem_bytes(int W, int K, int R, int rows) {
  const size_t P = size_t(rowconv_pitch(W, K)), Ht = size_t(sep_rows(rows, K));
  return (2 * size_t((2 * R * K + 3) & ~3) + (1 + size_t(R)) * Ht * P) * sizeof(float);
}

template <int K>
__global__ void __launch_bounds__(BAND_THREADS, 2) k_conv_sep_bands(const __grid_constant__ OneSeg src, int mode,
                                                                       int rows) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  __shared__ double red2[2 * (BAND_THREADS / 32)];
  __shared__ double band_sum[2];
  const PdlScope pdl;
  constexpr int c = (K - 1) / 2;
  const Seg& s = src.s;
  const int nb = int(cluster.num_blocks()), rank = int(cluster.block_rank());
  const int b = blockIdx.x / nb;
  const int H = s.H, W = s.W, HW = H * W, R = s.psf_rank;
  const int r0 = min(H, rank * rows), nr = min(H, r0 + rows) - r0;   // nr may be 0
  const SepLayout L = sep_layout(s, smem, rows);                      // local row li holds image row r0 - c + li
  const int P = L.P;
  float* work = s.work + size_t(b) * HW;
  const bool want_sim = (mode == MODE_SIM);
  const bool corr_only = (mode == MODE_CORR);
  const bool want_grad = (mode == MODE_GRAD) || corr_only;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;

  for (int i = threadIdx.x; i < 2 * R * K; i += blockDim.x) L.fac[i] = s.psf_sep[i];
  for (int i = threadIdx.x; i < R * K; i += blockDim.x) {
    const float u = s.psf_sep[(i / K) * 2 * K + i % K];
    L.tapu[i] = make_float2(u, u);
  }
  // the band's rows and halo rows of the input; rows outside the image, or
  // past the last halo row, are zero
  for (int li = wid; li < L.Ht; li += nw) {
    const int g = r0 - c + li;
    float* row = L.img + li * P;
    if (li < nr + K - 1 && g >= 0 && g < H) {
      for (int j = lane; j < W; j += 32) cp_async4(&row[j + c], &work[g * W + j]);
      for (int q = lane; q < P - W; q += 32) row[q < c ? q : W + q] = 0.f;
    } else {
      for (int j = lane; j < P; j += 32) row[j] = 0.f;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const int Wp2 = (W + 1) >> 1, nvu = ((nr + SEP_RV - 1) / SEP_RV) * Wp2;
  if (!corr_only) {
    sep_hpass<K, true, 0>(L.img, L, W, R);
    __syncthreads();
    float ll = 0.f, c2 = 0.f;
    for (int u = threadIdx.x; u < nvu; u += blockDim.x) {
      const int strip = u / Wp2, j = 2 * (u - strip * Wp2), i0 = strip * SEP_RV;
      const bool two = j + 1 < W;
      float2 m[SEP_RV];
      sep_vunit<K, true, 0>(L, R, i0, j, m);
#pragma unroll
      for (int o = 0; o < SEP_RV; ++o) {
        const int li = i0 + o;
        if (li >= nr) break;
        const int p = (r0 + li) * W + j;
        if (want_sim) {
          s.sim[size_t(b) * HW + p] = m[o].x;
          if (two) s.sim[size_t(b) * HW + p + 1] = m[o].y;
          continue;
        }
        const float g0 = pixel_terms(s, p, m[o].x, ll, c2);
        if (want_grad) L.img[(li + c) * P + j + c] = g0;
        if (two) {
          const float g1 = pixel_terms(s, p + 1, m[o].y, ll, c2);
          if (want_grad) L.img[(li + c) * P + j + 1 + c] = g1;
        }
      }
    }
    ll = warp_sum_f(ll);
    c2 = warp_sum_f(c2);
    if (lane == 0) {
      red2[2 * wid] = double(ll);
      red2[2 * wid + 1] = double(c2);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double Ls = 0.0, Cs = 0.0;
      for (int w = 0; w < nw; ++w) {
        Ls += red2[2 * w];
        Cs += red2[2 * w + 1];
      }
      band_sum[0] = Ls;
      band_sum[1] = Cs;
    }
    cluster.sync();   // every band's d log L / d M and sums are in its shared memory
    if (!want_sim && rank == 0 && threadIdx.x == 0) {
      double Ls = 0.0, Cs = 0.0;
      for (int r = 0; r < nb; ++r) {
        const double* bs = cluster.map_shared_rank(band_sum, r);
        Ls += bs[0];
        Cs += bs[1];
      }
      if (s.loglik) s.loglik[b] = -0.5 * Ls;
      if (s.chi2) s.chi2[b] = Cs;
    }
    if (want_grad) {
      // the halo rows of d log L / d M from the bands that own them
      for (int li = wid; li < nr + K - 1; li += nw) {
        if (li >= c && li < c + nr) continue;
        const int g = r0 - c + li;
        if (g < 0 || g >= H) continue;   // stays zero
        const int owner = g / rows;
        const float* orow = cluster.map_shared_rank(L.img, owner) + (g - owner * rows + c) * P + c;
        for (int j = lane; j < W; j += 32) L.img[li * P + j + c] = orow[j];
      }
    }
    cluster.sync();   // no block reads another's shared memory after this barrier
    if (!want_grad) return;
  } else {
    cluster.sync();   // every band holds its input before any band writes the work slot
  }
  sep_hpass<K, false, 0>(L.img, L, W, R);
  __syncthreads();
  const float inv_k2 = 1.0f / float(s.k * s.k);
  for (int u = threadIdx.x; u < nvu; u += blockDim.x) {
    const int strip = u / Wp2, j = 2 * (u - strip * Wp2), i0 = strip * SEP_RV;
    float2 m[SEP_RV];
    sep_vunit<K, false, 0>(L, R, i0, j, m);
#pragma unroll
    for (int o = 0; o < SEP_RV; ++o) {
      const int li = i0 + o;
      if (li >= nr) break;
      work[(r0 + li) * W + j] = m[o].x * inv_k2;
      if (j + 1 < W) work[(r0 + li) * W + j + 1] = m[o].y * inv_k2;
    }
  }
}

// ------------------------------------------------------------- k_final ----

// The FP64 factors of a vector's chain rule, from five reciprocals:
// b_n / n = 1.9992 - 0.3271 / n of the source and of the lens light, and
// 1 / thetaE, 1 / R_l, 1 / R_s.
struct ChainF {
  double ms, ml, ite, iRl, iRs;
};
// Parameter whose reciprocal is factor i of chain_factors.
__device__ __forceinline__ float recip_param(const float* pf, int i) {
  return pf[i == 0 ? 16 : i == 1 ? 9 : i == 2 ? 0 : i == 3 ? 8 : 15];
}
__device__ __forceinline__ ChainF chain_factors(const double* r) {
  ChainF f;
  f.ms = fma(-0.3271, r[0], 1.9992);
  f.ml = fma(-0.3271, r[1], 1.9992);
  f.ite = r[2];
  f.iRl = r[3];
  f.iRs = r[4];
  return f;
}

// The per-vector chain rule from the summed accumulators a[NACC], the
// parameters pf and the factors f (FP64 arithmetic): gradient entry j.
// Shared by the two k_final variants so that they give identical results.
__device__ __forceinline__ double chain_rule(int j, const double* a, const float* pf, const ChainF& f) {
  const double ln2 = 0.69314718055994530942;
  if (j < 8) return j == 0 ? f.ms * (double(pf[1]) - 1.0) * f.ite * a[A_THETAE] : f.ms * a[A_THETAE + j];
  const int l = j < 15 ? 0 : 1, k = j - (l == 0 ? 8 : 15);
  const double* c = a + (l == 0 ? A_L_R : A_S_R);
  const double m = l == 0 ? f.ml : f.ms;
  switch (k) {
    case 0: return m * (l == 0 ? f.iRl : f.iRs) * c[0];
    case 1: return -1.9992 * c[1] + m * ln2 * c[2];
    case 2: return -0.5 * m * c[3];
    case 3: return -0.5 * m * c[4];
    case 4: return m * c[5];
    case 5: return m * c[6];
    default: return c[7];
  }
}

// One thread per vector (calls whose vectors have one ray tile each).
// Block size of k_final (one thread per vector): one warp, so that a large
// batch's FP64 chain rule spreads over four times as many SMs as with
// FINAL_THREADS (60x60, B = 4096: 11.2 -> 10.7 us).
constexpr int FINAL1_THREADS = 32;

template <class Src>
__global__ void k_final(const __grid_constant__ Src src) {
  const PdlScope pdl;
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < src.nvec(); item += gridDim.x * blockDim.x) {
    int p;
    const Seg* s = src.vec_seg(item, p);
    const int b = slot_vector(*s, p);
    double* g = s->grad + size_t(b) * NPARAM;
    if (s->vc[p].nterms < 0) {
      for (int i = 0; i < NPARAM; ++i) g[i] = nan("");
      continue;
    }
    double a[NACC];
    for (int i = 0; i < NACC; ++i) a[i] = 0.0;
    const double* part = s->partial + size_t(b) * s->ntiles * NACC;
    for (int t = 0; t < s->ntiles; ++t)
      for (int i = 0; i < NACC; ++i) a[i] += part[t * NACC + i];
    const float* pf = s->params + size_t(b) * NPARAM;
    double r[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) r[i] = 1.0 / double(recip_param(pf, i));
    const ChainF f = chain_factors(r);
    for (int j = 0; j < NPARAM; ++j) g[j] = chain_rule(j, a, pf, f);
  }
}

// One warp per vector (many tiles per vector, i.e. small batches): lane i <
// NACC sums accumulator i over the tiles in tile order, lane j < NPARAM
// applies the chain rule for entry j.
template <class Src>
__global__ void k_final_warp(const __grid_constant__ Src src) {
  __shared__ double sa[FINAL_THREADS / 32][NACC];
  const PdlScope pdl;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  for (int item = blockIdx.x * wpb + w; item < src.nvec(); item += gridDim.x * wpb) {
    int p;
    const Seg* s = src.vec_seg(item, p);
    const int b = slot_vector(*s, p);
    double* g = s->grad + size_t(b) * NPARAM;
    if (s->vc[p].nterms < 0) {   // warp-uniform
      if (lane < NPARAM) g[lane] = nan("");
      continue;
    }
    if (lane < NACC) {
      // eight loads in flight, then added in tile order (the same sum as k_final)
      const double* part = s->partial + size_t(b) * s->ntiles * NACC + lane;
      const int nt = s->ntiles;
      double acc = 0.0;
      int t = 0;
      for (; t + 8 <= nt; t += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = part[size_t(t + u) * NACC];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u];
      }
      for (; t < nt; ++t) acc += part[size_t(t) * NACC];
      sa[w][lane] = acc;
    }
    __syncwarp();
    const float* pf = s->params + size_t(b) * NPARAM;
    // lanes 0..4 take the five divisions at once; every lane receives them
    const double rl = lane < 5 ? 1.0 / double(recip_param(pf, lane)) : 0.0;
    double r[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) r[i] = __shfl_sync(0xffffffffu, rl, i);
    const ChainF f = chain_factors(r);
    if (lane < NPARAM) g[lane] = chain_rule(lane, sa[w], pf, f);
    __syncwarp();
  }
}

// ------------------------------------------------------------- launch -----

// Guards the cached dynamic shared-memory limits of the launch helpers: a
// thread must not launch on a limit another thread has recorded but not yet set.
static std::mutex g_attr_mutex;

static std::atomic<int> g_num_sms{0};

static int num_sms() {
  int n = g_num_sms.load(std::memory_order_relaxed);
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
    g_num_sms.store(n, std::memory_order_relaxed);
  }
  return n;
}

// Convolution classes: (PSF side, strip rows, threads). Class 2 takes any odd side.
struct ConvClass {
  int K, R, NT;
};
static constexpr ConvClass kConvClasses[3] = {{11, 16, 256}, {21, 16, 256}, {0, 8, 128}};  // see launch_conv_class

int conv_class(int K) { return K == 11 ? 0 : (K == 21 ? 1 : 2); }

size_t conv_smem_bytes(int H, int W, int K, bool two_buf) {
  if (kConvClasses[conv_class(K)].K > 0) {   // row-strip layout (conv_vector_rows)
    const size_t KP = size_t((K + 3) & ~3), P = size_t(rowconv_pitch(W, K));
    return (2 * size_t(K) * KP + (size_t(H) + K - 1) * P + (two_buf ? size_t(H) * P : 0)) * sizeof(float);
  }
  const int R = kConvClasses[conv_class(K)].R;
  const int nstrip = (H + R - 1) / R;
  const size_t Hp = size_t(nstrip) * R + K - 1, Wp = size_t(W) + K - 1;
  return (2 * size_t((K * K + 3) & ~3) + (two_buf ? 2 : 1) * Hp * Wp) * sizeof(float);
}

bool conv_two_buf(int H, int W, int K) { return conv_smem_bytes(H, W, K, true) <= CONV_TWO_BUF_MAX_SMEM; }

size_t conv_sep_smem_bytes(int H, int W, int K, int R) {
  const size_t P = size_t(rowconv_pitch(W, K)), Ht = size_t(sep_rows(H, K));
  return (2 * size_t((2 * R * K + 3) & ~3) + (1 + size_t(R)) * Ht * P) * sizeof(float);
}

// 2 K R multiply-adds per pixel and pass against K^2, with a pass of
// shared-memory traffic per term: worth it at R <= K / 4
static bool conv_sep_worth(int K, int R) { return R > 0 && 4 * R <= K && (K == 11 || K == 21); }

bool conv_sep_ok(int H, int W, int K, int R) {
  return conv_sep_worth(K, R) && conv_sep_smem_bytes(H, W, K, R) <= CONV_TWO_BUF_MAX_SMEM;
}

// Row bands of the separable cluster convolution: at most 8 (a portable
// cluster) of at least max(16, (K - 1) / 2) rows, so that a band's halo rows
// come from its two neighbours. small: a batch below half as many vectors
// as SMs, up to 2 SMs / B bands of at least 2 (K - 1) rows (up to two
// blocks per SM over the call); else the fewest bands whose blocks fit two
// per SM, or one. Returns the band count (0: none) and the rows per band.
static int sep_band_plan(int H, int W, int K, int R, bool small, int B, int* rows_out) {
  const int min_rows = (K - 1) / 2 > 16 ? (K - 1) / 2 : 16;
  int best = 0, best_rows = 0;
  if (small) {
    // bands of at least 2 (K - 1) rows: thinner ones spend more on the halo
    // rows' horizontal passes than the extra blocks gain
    const int small_rows = 2 * (K - 1) > min_rows ? 2 * (K - 1) : min_rows;
    int nb = 2 * num_sms() / (B > 0 ? B : 1);
    if (nb > 8) nb = 8;
    while (nb > 1 && (H + nb - 1) / nb < small_rows) --nb;
    const int rows = (H + nb - 1) / nb;
    if (nb >= 2 && conv_sep_band_smem_bytes(W, K, R, rows) <= CONV_TWO_BUF_MAX_SMEM) best = nb, best_rows = rows;
  } else {
    // two blocks of 112 KB (and their reserved shared memory) fit an SM's 228 KB
    for (const size_t cap : {size_t(112 * 1024), size_t(CONV_TWO_BUF_MAX_SMEM)}) {
      for (int nb = 2; nb <= 8 && best == 0; ++nb) {
        const int rows = (H + nb - 1) / nb;
        if (rows < min_rows) break;
        if (conv_sep_band_smem_bytes(W, K, R, rows) <= cap) best = nb, best_rows = rows;
      }
      if (best) break;
    }
  }
  *rows_out = best_rows;
  return best;
}

bool conv_sep_any(int H, int W, int K, int R) {
  int rows;
  return conv_sep_ok(H, W, K, R) || (conv_sep_worth(K, R) && sep_band_plan(H, W, K, R, false, 0, &rows) > 0);
}

size_t seg_conv_smem(const Seg& g) {
  return g.conv_sep ? conv_sep_smem_bytes(g.H, g.W, g.K, g.psf_rank) : conv_smem_bytes(g.H, g.W, g.K, g.conv_two_buf != 0);
}

// Ray tiles of at most this many rays take the three-blocks-per-SM adjoint.
constexpr long long ADJ_SHORT_TILE_RAYS = 32768;

// Resident blocks per SM of the forward ray kernel (occupancy query, cached;
// its launch bound if the query fails, e.g. without a GPU).
static int fwd_blocks_per_sm() {
  static std::atomic<int> cached{0};
  int n = cached.load(std::memory_order_relaxed);
  if (n == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ray_fwd<OneSeg>, FWD_THREADS, 0) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = GL_FWD_MINB;
    }
    cached.store(n, std::memory_order_relaxed);
  }
  return n;
}

// Tiling of a B-vector call's rays: the tile count that minimises a model of
// the two ray kernels' time, waves x (pixels per tile + a fixed per-tile
// cost of 64 pixels), the forward kernel at its resident blocks per SM and
// the adjoint, 2.4 times the forward's cost per ray (measured at 60 x 60,
// k = 2), at two or three blocks per SM (a three-block wave takes 3/2.054 of
// a two-block wave: a block's time grows with the blocks sharing its SM, and
// three share 1.027x the work of two; three only for tiles of at most
// ADJ_SHORT_TILE_RAYS rays, whose spills cost little). Tiles keep at least
// 8 rays per thread of a 256-thread block; ties go to fewer tiles. Below
// one vector per SM the forward's waves weigh half: there they are partly
// filled, and its blocks, sharing an SM with fewer others, finish sooner
// than the model's full wave. 50 vectors of 80 x 80, k = 2, then take 9
// tiles (one three-block adjoint wave) instead of 12 (46.9 -> 44.1 us a
// call near one mode, 56.7 -> 54.0 us for vectors drawn from the prior);
// 100 x 100, k = 4: 145.5 -> 145.0 us. Larger batches keep weight 1: with
// half, 300 vectors from the prior took 2 tiles instead of 5 (178 -> 204 us;
// the model does not see a batch's spread of per-vector cost).
struct TilePlan {
  int ntiles, tile_pix;
  bool adj3;
};

static TilePlan plan_rays(int B, int H, int W, int k) {
  const int HW = H * W;
  TilePlan best{1, HW, false};
  if (B <= 0 || HW <= 0) return best;
  const long long rays = (long long)HW * k * k;
  long long max_nt = (rays + RAY_THREADS * 8 - 1) / (RAY_THREADS * 8);
  if (max_nt > HW) max_nt = HW;
  if (max_nt < 1) max_nt = 1;
  const double sms = num_sms(), fwd_slots = sms * fwd_blocks_per_sm();
  const double wf = B < sms ? 0.5 : 1.0;   // weight of the forward's waves
  double best_cost = 0.0;
  for (long long nt = 1; nt <= max_nt; ++nt) {
    const int tp = int((HW + nt - 1) / nt);
    const int ntt = (HW + tp - 1) / tp;
    if (ntt != nt) continue;   // the same tiling as a smaller count
    const double items = double(B) * ntt, px = tp + 64.0;
    const double fwd = std::ceil(items / fwd_slots) * px;
    const double adj2 = std::ceil(items / (2 * sms)) * px;
    const bool short_tile = (long long)tp * k * k <= ADJ_SHORT_TILE_RAYS;
    const double adj3 = short_tile ? std::ceil(items / (3 * sms)) * px * (3.0 / 2.054) : 1e300;
    const double cost = wf * fwd + 2.4 * (adj3 < adj2 ? adj3 : adj2);
    if (nt == 1 || cost < best_cost * (1.0 - 1e-9)) {
      best_cost = cost;
      best = TilePlan{ntt, tp, adj3 < adj2};
    }
  }
  return best;
}

void plan_tiles(int B, int H, int W, int k, int* ntiles, int* tile_pix) {
  const TilePlan p = plan_rays(B, H, W, k);
  *ntiles = p.ntiles;
  *tile_pix = p.tile_pix;
}

// Blocks of a convolution kernel resident on the whole GPU at a dynamic
// shared-memory size (occupancy query, cached per kernel and size; the
// grouped path warms it before a graph capture).
template <int K, int R, int NT, int MINB, class Src>
static cudaError_t conv_resident(size_t smem, int* resident) {
  static std::map<size_t, int> per_sm;   // by dynamic shared memory
  std::lock_guard<std::mutex> lock(g_attr_mutex);
  auto it = per_sm.find(smem);
  if (it == per_sm.end()) {
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_conv<K, R, NT, MINB, Src>, NT, smem);
    if (e != cudaSuccess) return e;
    it = per_sm.emplace(smem, n > 0 ? n : 1).first;
  }
  *resident = num_sms() * it->second;
  return cudaSuccess;
}

// Launch with programmatic stream serialization (see pdl_begin): the kernel
// may be scheduled while its predecessor in the stream drains.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <int K, int R, int NT, int MINB, class Src>
static cudaError_t launch_conv(const Src& src, int nitems, size_t smem, int mode, cudaStream_t st, bool persistent) {
  static size_t attr = 48 * 1024;
  {
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (smem > attr) {
      cudaError_t e = cudaFuncSetAttribute(k_conv<K, R, NT, MINB, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(smem));
      if (e != cudaSuccess) return e;
      attr = smem;
    }
  }
  int grid = nitems;
  if (persistent) {
    // as many blocks as fit on the GPU at once: with a static split of the
    // items, blocks beyond that would start only after others have finished
    // their whole share
    int resident = 0;
    cudaError_t e = conv_resident<K, R, NT, MINB, Src>(smem, &resident);
    if (e != cudaSuccess) return e;
    grid = grid < resident ? grid : resident;
  }
  return launch_pdl(k_conv<K, R, NT, MINB, Src>, unsigned(grid), NT, smem, st, src, mode);
}

// wide: 512-thread blocks for calls with fewer vectors than SMs (one vector's
// work spread over 16 warps) and for blocks that hold an SM's shared memory
// alone (CONV_WIDE_MIN_SMEM). Every pixel's model value and d log L / d M is
// computed by one thread whatever the width, so gradients are the same bits;
// log L and chi^2 are summed in a width-dependent order (last FP32 bits).
template <class Src>
static cudaError_t launch_conv_class(int cls, const Src& src, int nitems, size_t smem, int mode, cudaStream_t st,
                                     bool persistent, bool wide = false) {
  switch (cls) {
    case 0:
      return wide ? launch_conv<11, 16, 512, 1>(src, nitems, smem, mode, st, persistent)
                  : launch_conv<11, 16, 256, 3>(src, nitems, smem, mode, st, persistent);
    case 1:
      return wide ? launch_conv<21, 16, 512, 1>(src, nitems, smem, mode, st, persistent)
                  : launch_conv<21, 16, 256, 1>(src, nitems, smem, mode, st, persistent);
    default: return launch_conv<0, 8, 128, 4>(src, nitems, smem, mode, st, persistent);
  }
}

template <int K, int NT, int MINB>
static cudaError_t launch_conv_sep(const OneSeg& src, int nitems, size_t smem, int mode, cudaStream_t st) {
  static size_t attr = 48 * 1024;
  {
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (smem > attr) {
      cudaError_t e = cudaFuncSetAttribute(k_conv_sep<K, NT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(smem));
      if (e != cudaSuccess) return e;
      attr = smem;
    }
  }
  // at most the blocks resident at once: each prepares its factors and halo
  // once and then takes every gridDim-th vector
  static std::map<size_t, int> per_sm;   // by dynamic shared memory
  int resident;
  {
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    auto it = per_sm.find(smem);
    if (it == per_sm.end()) {
      int n = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_conv_sep<K, NT, MINB>, NT, smem);
      if (e != cudaSuccess) return e;
      it = per_sm.emplace(smem, n > 0 ? n : 1).first;
    }
    resident = num_sms() * it->second;
  }
  const int grid = nitems < resident ? nitems : resident;
  return launch_pdl(k_conv_sep<K, NT, MINB>, unsigned(grid), NT, smem, st, src, mode);
}

// The convolution of a single-system call over nitems vectors: the
// separable kernel when the segment takes it, else its PSF-size class.
static cudaError_t launch_conv_one(const OneSeg& src, int nitems, int mode, cudaStream_t st, bool wide) {
  const Seg& s = src.s;
  const size_t smem = seg_conv_smem(s);
  if (s.conv_sep) {
    if (s.K == 11)
      return wide ? launch_conv_sep<11, 512, 1>(src, nitems, smem, mode, st)
                  : launch_conv_sep<11, 256, 4>(src, nitems, smem, mode, st);
    return wide ? launch_conv_sep<21, 512, 1>(src, nitems, smem, mode, st)
                : launch_conv_sep<21, 256, 3>(src, nitems, smem, mode, st);
  }
  return launch_conv_class(conv_class(s.K), src, nitems, smem, mode, st, false, wide || smem > CONV_WIDE_MIN_SMEM);
}

// Row bands for the cluster convolution of a B-vector call (0: one block per
// vector instead). Bands only below half as many vectors as SMs: up to two
// blocks per SM, at most 8 per vector (a portable cluster), each at least
// max(16, (K - 1) / 2) rows and within CONV_TWO_BUF_MAX_SMEM of shared memory.
static int conv_bands(int B, int H, int W, int K) {
  if ((K != 11 && K != 21) || B < 1 || 2 * B > num_sms()) return 0;
  int nb = 2 * num_sms() / B;
  if (nb > 8) nb = 8;
  const int min_rows = (K - 1) / 2 > 16 ? (K - 1) / 2 : 16;
  while (nb > 1 && (H + nb - 1) / nb < min_rows) --nb;
  if (nb < 2 || conv_band_smem_bytes(W, K, (H + nb - 1) / nb) > CONV_TWO_BUF_MAX_SMEM) return 0;
  return nb;
}

template <int K>
static cudaError_t launch_conv_bands(const OneSeg& src, int nb, int mode, cudaStream_t st) {
  static size_t attr = 48 * 1024;
  const int rows = (src.s.H + nb - 1) / nb;
  const size_t smem = conv_band_smem_bytes(src.s.W, K, rows);
  {
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (smem > attr) {
      cudaError_t e = cudaFuncSetAttribute(k_conv_bands<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
      attr = smem;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(src.s.B) * unsigned(nb));
  cfg.blockDim = dim3(BAND_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = unsigned(nb);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_conv_bands<K>, src, mode, rows);
}

template <int K>
static cudaError_t launch_conv_sep_bands(const OneSeg& src, int nb, int rows, int mode, cudaStream_t st) {
  static size_t attr = 48 * 1024;
  const size_t smem = conv_sep_band_smem_bytes(src.s.W, K, src.s.psf_rank, rows);
  {
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (smem > attr) {
      cudaError_t e = cudaFuncSetAttribute(k_conv_sep_bands<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
      attr = smem;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(src.s.B) * unsigned(nb));
  cfg.blockDim = dim3(BAND_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = unsigned(nb);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_conv_sep_bands<K>, src, mode, rows);
}

// Vectors at or above this count are taken longest series first (k_order).
// Graph-replayed calls at 80 x 80, k = 2, vectors drawn from the prior, in
// random order against heaviest first: 300 vectors 179.6 -> 163.9 us, 1000
// vectors 478.3 -> 465.2 us; 60 x 60, B = 4096: 958.9 -> 939.6 us. Below
// it the sort's launch is not repaid (a 50-vector call near one mode).
static bool ray_order_pays(const Seg& s) { return s.B >= num_sms() && s.H * s.W >= 2; }

// k_order before k_setup, for single-segment calls that take their vectors
// in order.
static bool takes_order(const OneSeg& src) { return src.s.ray_order != 0; }
template <class Src>
static bool takes_order(const Src&) { return false; }
static cudaError_t launch_order(const OneSeg& src, int stage, cudaStream_t st) {
  if (stage == 0)
    return launch_pdl(k_keys, unsigned((src.s.B + KEYS_THREADS - 1) / KEYS_THREADS), KEYS_THREADS, 0, st, src);
  return launch_pdl(k_order, 1u, ORDER_THREADS, 0, st, src);
}
template <class Src>
static cudaError_t launch_order(const Src&, int, cudaStream_t) { return cudaErrorInvalidValue; }

template <class Src>
static cudaError_t run_rays(const Src& src, int nvec, int nray, bool fwd, bool adj_final, cudaStream_t st,
                            Hooks* hooks, bool persistent, bool one_tile = false, bool fwd_rays = true,
                            bool short_tiles = false) {
  const int sms = num_sms();
  cudaError_t e;
  const int vthreads = SETUP_THREADS, wpb = vthreads / 32 - 2;
  int sgrid = (nvec + wpb - 1) / wpb;
  int fgrid = (nvec + FINAL1_THREADS - 1) / FINAL1_THREADS;
  int wgrid = (nvec + FINAL_THREADS / 32 - 1) / (FINAL_THREADS / 32);
  int rgrid = nray;
  if (persistent) {
    sgrid = sgrid < sms * 4 ? sgrid : sms * 4;
    fgrid = fgrid < sms * 4 ? fgrid : sms * 4;
    wgrid = wgrid < sms * 4 ? wgrid : sms * 4;
    rgrid = rgrid < sms * 4 ? rgrid : sms * 4;
  }
  if (fwd) {
    if (takes_order(src)) {
      for (int stage = 0; stage < 2; ++stage) {   // k_keys, k_order
        hooks->before(GL_K_ORDER, st);
        e = launch_order(src, stage, st);
        const cudaError_t h = hooks->after(GL_K_ORDER, st);
        if (e != cudaSuccess || (e = h) != cudaSuccess) return e;
      }
    }
    hooks->before(GL_K_SETUP, st);
    e = launch_pdl(k_setup<Src>, unsigned(sgrid), vthreads, 0, st, src);
    cudaError_t h = hooks->after(GL_K_SETUP, st);
    if (e != cudaSuccess || (e = h) != cudaSuccess) return e;
    if (!fwd_rays) return cudaSuccess;   // setup only (the correlation-only gradient)
    hooks->before(GL_K_RAY_FWD, st);
    e = launch_pdl(k_ray_fwd<Src>, unsigned(rgrid), FWD_THREADS, 0, st, src);
    h = hooks->after(GL_K_RAY_FWD, st);
    return e != cudaSuccess ? e : h;
  }
  if (adj_final) {
    hooks->before(GL_K_RAY_ADJ, st);
    if (short_tiles)
      e = launch_pdl(k_ray_adj<Src, 3>, unsigned(rgrid), ADJ_THREADS, 0, st, src);
    else
      e = launch_pdl(k_ray_adj<Src>, unsigned(rgrid), ADJ_THREADS, 0, st, src);
    cudaError_t h = hooks->after(GL_K_RAY_ADJ, st);
    if (e != cudaSuccess || (e = h) != cudaSuccess) return e;
    hooks->before(GL_K_FINAL, st);
    if (one_tile)
      e = launch_pdl(k_final<Src>, unsigned(fgrid), FINAL1_THREADS, 0, st, src);
    else
      e = launch_pdl(k_final_warp<Src>, unsigned(wgrid), FINAL_THREADS, 0, st, src);
    h = hooks->after(GL_K_FINAL, st);
    return e != cudaSuccess ? e : h;
  }
  return cudaSuccess;
}

cudaError_t launch_one(const Seg& s0, int mode, cudaStream_t st, Hooks* hooks) {
  if (s0.B <= 0) return cudaSuccess;
  Seg s = s0;
  // the key and slot arrays take 2 B ints of the work buffer, which in
  // MODE_CORR already holds the vectors' d log L / d M
  s.ray_order = mode != MODE_CORR && ray_order_pays(s) ? 1 : 0;
  OneSeg src{s};
  cudaError_t e = run_rays(src, s.B, s.B * s.ntiles, true, false, st, hooks, false, false, mode != MODE_CORR);
  if (e != cudaSuccess) return e;
  hooks->before(GL_K_CONV, st);
  // a separable PSF: the whole image in one block, or row bands over a
  // cluster (small batches, and images whose buffers do not fit one block);
  // else the 2-D stencil, in bands for small batches
  int rows = 0;
  const bool small = 2 * s.B <= num_sms();
  const int sb = s.psf_rank > 0 && (small || !s.conv_sep) ? sep_band_plan(s.H, s.W, s.K, s.psf_rank, small, s.B, &rows) : 0;
  const int nb = (sb > 0 || mode == MODE_CORR || s.conv_sep) ? 0 : conv_bands(s.B, s.H, s.W, s.K);
  if (sb > 0)
    e = s.K == 11 ? launch_conv_sep_bands<11>(src, sb, rows, mode, st)
                  : launch_conv_sep_bands<21>(src, sb, rows, mode, st);
  else if (nb > 0)
    e = s.K == 11 ? launch_conv_bands<11>(src, nb, mode, st) : launch_conv_bands<21>(src, nb, mode, st);
  else
    e = launch_conv_one(src, s.B, mode, st, s.B < num_sms());
  if (e != cudaSuccess) return e;
  if ((e = hooks->after(GL_K_CONV, st)) != cudaSuccess) return e;
  if (mode != MODE_GRAD && mode != MODE_CORR) return cudaSuccess;
  // the adjoint's blocks per SM as the tile plan chose them (plan_rays)
  const TilePlan tp = plan_rays(s.B, s.H, s.W, s.k);
  const bool three = tp.adj3 && tp.ntiles == s.ntiles && tp.tile_pix == s.tile_pix;
  return run_rays(src, s.B, s.B * s.ntiles, false, true, st, hooks, false, s.ntiles == 1, true, three);
}

cudaError_t launch_basis(const Seg& s, cudaStream_t st, Hooks* hooks) {
  if (s.B <= 0) return cudaSuccess;
  OneSeg src{s};
  cudaError_t e = run_rays(src, s.B, s.B * s.ntiles, true, false, st, hooks, false, false, false);   // setup
  if (e != cudaSuccess) return e;
  hooks->before(GL_K_RAY_FWD, st);
  if ((e = launch_pdl(k_ray_fwd_basis<OneSeg>, unsigned(s.B * s.ntiles), FWD_THREADS, 0, st, src)) != cudaSuccess)
    return e;
  if ((e = hooks->after(GL_K_RAY_FWD, st)) != cudaSuccess) return e;
  Seg c = s;
  c.B = 2 * s.B;   // the convolution takes the two images of every vector as vectors of their own
  OneSeg csrc{c};
  hooks->before(GL_K_CONV, st);
  e = launch_conv_one(csrc, c.B, MODE_SIM, st, c.B < num_sms());
  if (e != cudaSuccess) return e;
  return hooks->after(GL_K_CONV, st);
}

cudaError_t launch_table(const Seg* d_segs, int nseg, int vec_total, int ray_total, const ConvRun* conv, int nconv,
                         int mode, cudaStream_t st, Hooks* hooks) {
  if (vec_total <= 0) return cudaSuccess;
  SegTable src{d_segs, nseg, vec_total, ray_total, 0, nseg, vec_total};
  cudaError_t e = run_rays(src, vec_total, ray_total, true, false, st, hooks, true);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < nconv; ++i) {
    SegTable cs = src;
    cs.conv_first = conv[i].first;
    cs.conv_nseg = conv[i].nseg;
    cs.conv_total = conv[i].nitems;
    hooks->before(GL_K_CONV, st);
    e = launch_conv_class(conv[i].cls, cs, conv[i].nitems, conv[i].smem, mode, st, true,
                          conv[i].smem > CONV_WIDE_MIN_SMEM);
    if (e != cudaSuccess) return e;
    if ((e = hooks->after(GL_K_CONV, st)) != cudaSuccess) return e;
  }
  if (mode != MODE_GRAD) return cudaSuccess;
  return run_rays(src, vec_total, ray_total, false, true, st, hooks, true);
}

// Grouped launch whose counts live in device memory: fixed persistent grids,
// every convolution class launched (an empty class exits at once). Safe to
// capture into a CUDA graph; conv_smem[c] is the dynamic shared memory of
// class c and must cover every segment of that class.
template <int K, int R, int NT, int MINB>
static cudaError_t set_devtable_attr(size_t smem) {
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_conv<K, R, NT, MINB, DevTable>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  int resident = 0;   // the occupancy query before any capture
  return conv_resident<K, R, NT, MINB, DevTable>(smem, &resident);
}

cudaError_t prepare_devtable(const size_t* conv_smem) {
  cudaError_t e;
  (void)fwd_blocks_per_sm();   // the occupancy query before any capture
  e = conv_smem[0] > CONV_WIDE_MIN_SMEM ? set_devtable_attr<11, 16, 512, 1>(conv_smem[0])
                                        : set_devtable_attr<11, 16, 256, 3>(conv_smem[0]);
  if (e != cudaSuccess) return e;
  e = conv_smem[1] > CONV_WIDE_MIN_SMEM ? set_devtable_attr<21, 16, 512, 1>(conv_smem[1])
                                        : set_devtable_attr<21, 16, 256, 1>(conv_smem[1]);
  if (e != cudaSuccess) return e;
  return set_devtable_attr<0, 8, 128, 4>(conv_smem[2]);
}

cudaError_t launch_devtable(const TableHdr* d_hdr, const Seg* d_segs, const size_t* conv_smem, cudaStream_t st,
                            Hooks* hooks) {
  const int sms = num_sms();
  cudaError_t e;
  DevTable src{d_hdr, d_segs, 0};
  hooks->before(GL_K_SETUP, st);
  if ((e = launch_pdl(k_setup<DevTable>, unsigned(sms * 2), SETUP_THREADS, 0, st, src)) != cudaSuccess) return e;
  if ((e = hooks->after(GL_K_SETUP, st)) != cudaSuccess) return e;
  hooks->before(GL_K_RAY_FWD, st);
  if ((e = launch_pdl(k_ray_fwd<DevTable>, unsigned(sms * fwd_blocks_per_sm()), FWD_THREADS, 0, st, src)) !=
      cudaSuccess)
    return e;
  if ((e = hooks->after(GL_K_RAY_FWD, st)) != cudaSuccess) return e;
  for (int c = 0; c < N_CONV_CLASSES; ++c) {
    DevTable cs{d_hdr, d_segs, c};
    hooks->before(GL_K_CONV, st);
    e = launch_conv_class(c, cs, 1 << 30, conv_smem[c], MODE_GRAD, st, true, conv_smem[c] > CONV_WIDE_MIN_SMEM);
    if (e != cudaSuccess) return e;
    if ((e = hooks->after(GL_K_CONV, st)) != cudaSuccess) return e;
  }
  hooks->before(GL_K_RAY_ADJ, st);
  if ((e = launch_pdl(k_ray_adj<DevTable>, unsigned(sms * GL_ADJ_MINB), ADJ_THREADS, 0, st, src)) != cudaSuccess)
    return e;
  if ((e = hooks->after(GL_K_RAY_ADJ, st)) != cudaSuccess) return e;
  hooks->before(GL_K_FINAL, st);
  if ((e = launch_pdl(k_final_warp<DevTable>, unsigned(sms * 4), FINAL_THREADS, 0, st, src)) != cudaSuccess) return e;
  return hooks->after(GL_K_FINAL, st);
}

}  // namespace gl
