// Travel-time matrices built on the device from location coordinates (Eq. e1,
// Section 3): for every instance of a batch and every vehicle type t,
//   T[t][i][j] = rint(dist_km(i, j) / speed_kmh[t] * 60)   (integer minutes, half to even)
// with the Haversine distance of Eq. e1 on (latitude, longitude) in degrees, or the
// Euclidean distance on (x, y) kilometres. float64 throughout, as the paper's Python.
//
// The Euclidean path rounds every operation explicitly (no contraction into fused
// multiply-adds), in the order subtract, square, add, square root, divide, multiply, so
// it returns the same integers as any IEEE float64 evaluation of that expression. The
// Haversine path calls the device sine, cosine and arcsine, which may differ from a host
// library in the last bits; the integer result then differs only where the exact time
// lies within a few ulps of a half minute.
//
// Most entries are decided in float32, with float64 only where float32 cannot vouch for
// the integer: rint changes value only at half minutes, so when the float32 time lies
// farther from the nearest half minute than a bound on its error, it rounds to the same
// integer as the float64 expression (whose own error is far smaller).
// Bounds on the float32 time t (every float32 value of a coordinate is off by at most
// 2^-24 of its magnitude):
//   Euclidean  coordinates staged as float32; the differences add at most 2^-24 of the
//              sum of the four magnitudes, then differences, squares, sum, square root
//              and the product with a rounded 60 / speed add below 6 * 2^-24 relative with
//              a correctly rounded root, 10 * 2^-24 with the root as a * rsqrtf(a) (rsqrtf
//              within 2 ulp, CUDA's documented bound, plus one rounded product); screened
//              at 2e-6 t + (60 / speed) 2^-20 S + 1e-6, S the instance's largest |x| + |y|;
//   Haversine  angles staged as float pairs hi + lo (lo = float(v - hi)), so a difference
//              (hi_i - hi_j) + (lo_i - lo_j) is within 2 * 2^-24 of itself plus 2^-47 of
//              the magnitudes; half-angle differences, sinf (2 ulp), squares, cos(phi)
//              staged from float64, sum, square root and asinf (2 ulp) with its condition
//              number below 1.9 for sqrt(a) <= 0.9 (larger values go to float64 outright)
//              add below 1.8e-6 relative; screened at 8e-6 t + (60 / speed) 2 r 2^-40
//              (sum of |angles|) + 1e-5.
// Times of 2^22 minutes or more also go to float64 (small instances: every entry of an
// instance whose largest possible time, 2 S * 60 / speed or pi r * 60 / speed, is not
// below 2^22, through an infinite tolerance). The float32 time is rounded by adding
// and subtracting 1.5 * 2^23: for 0 <= t < 2^22 the sum lies in [2^23, 2^24), where the
// float32 spacing is 1, so the addition itself rounds t half to even, the integer is the
// sum's low mantissa bits, and t minus the rounded value is exact (Sterbenz), which gives
// the distance to the nearest half minute without a conversion instruction. The float64
// path is the expression above, on the original float64 coordinates. Lanes that need it
// queue (row, column, type) in shared memory, so float64 work runs on full warps and
// follows the number of such entries: large instances keep a queue per warp, drained when
// it fills and at the end of the instance; small instances one queue per CTA, drained
// after the pairs by as many warps as it has entries (one, as a rule), entries beyond its
// capacity computed where they arise.
//
// One CTA per instance (grid-stride over instances); the instance's coordinates are
// staged once in shared memory (angles in radians and cos(phi) for Haversine). Two
// kernels share a batch, each skipping the other's instances:
//   Small instances (n_types * L^2 + 3 <= kOut words, L <= kSmallLoc: L <= 55 for two
//   types, 78 for one) are built whole in shared memory by 128-thread CTAs, eight per SM.
//   Both distances are symmetric in every rounded operation (x_i - x_j = -(x_j - x_i)
//   exactly, products commute), so each unordered pair i <= j is evaluated once and
//   written to (i, j) and (j, i). The L (L + 1) / 2 pairs are numbered row by row with row
//   i folded onto row L - 1 - i (L + 1 pairs per folded row), so the threads take
//   consecutive numbers with no idle lanes at row ends. The finished matrices, contiguous
//   in the output, leave by one bulk copy (cp.async.bulk, shared to global) on their
//   16-byte aligned middle and plain stores on the at most 3 + 3 words around it; the
//   next instance is staged while that copy runs and waits only for its reads of shared
//   memory, before its first write of the matrix.
//   Larger instances: 256-thread CTAs, warps take rows, lanes take columns, so a row's
//   writes are contiguous. An instance with more locations than the stage holds goes
//   through float64 alone.
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#include "asched.h"
#include "nvtx_range.h"

namespace {

constexpr int kStageLocations = 2048;  // large instances: 5 floats per location, 40 KB of shared memory
constexpr int kWarps = 8;              // large-instance CTAs: 8 warps, 4 per SM
constexpr int kThreads = kWarps * 32;
constexpr int kQueue = 128;            // deferred float64 entries per warp (large instances)
constexpr int kSmallThreads = 128;     // small-instance CTAs: 4 warps, 8 per SM
constexpr int kSmallLoc = 80;          // locations of an instance built in shared memory
constexpr int kOut = 6144;             // int32 words of that instance's matrices
constexpr int kSmallQueue = 256;       // deferred float64 entries per CTA (small instances)

__host__ __device__ __forceinline__ bool is_small(int L, int nt) {
  return L <= kSmallLoc && nt * L * L + 3 <= kOut;
}

struct MParams {
  int32_t B, nt, metric;
  double speed[2];
  float k32[2];  // float(60 / speed)
  float rel_hav;  // Haversine screen: 8e-6, or infinity if a time may reach 2^22 minutes
  double two_r, deg;
  const int32_t* loc_off;
  const int64_t* travel_off;
  const double* coords;
  int32_t* travel;
  int32_t* status;
};

struct Stage {  // structure of arrays: hi and lo of both coordinates, cos(phi)
  float xh[kStageLocations], xl[kStageLocations], yh[kStageLocations], yl[kStageLocations];
  float cphi[kStageLocations];
};

struct SmallStage {  // 26,816 bytes: with the queue, eight CTAs fit one SM
  float4 hl[kSmallLoc];     // (x hi, y hi, x lo, y lo)
  float cphi[kSmallLoc];    // float(cos(phi))
  double cos64[kSmallLoc];  // cos(phi) in float64, as the definition computes it
  int32_t out[kOut];        // the instance's matrices, offset so that they share the output's 16-byte phase
};
static_assert(offsetof(SmallStage, out) % 16 == 0, "the bulk copy reads out at 16-byte boundaries");
static_assert(kSmallLoc <= kSmallThreads, "one location per thread when staging");

__device__ __forceinline__ double euclid(double xi, double yi, double xj, double yj) {
  const double dx = __dsub_rn(xi, xj), dy = __dsub_rn(yi, yj);
  return __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

// Eq. e1 with the cosines of both latitudes given (each equals cos(lat * deg) bit for bit).
__device__ __forceinline__ double haversine(double lati, double loni, double latj, double lonj, double ci, double cj,
                                            double two_r, double deg) {
  const double phi_i = __dmul_rn(lati, deg), phi_j = __dmul_rn(latj, deg);
  const double s1 = sin(__dmul_rn(__dsub_rn(phi_i, phi_j), 0.5));
  const double s2 = sin(__dmul_rn(__dsub_rn(__dmul_rn(loni, deg), __dmul_rn(lonj, deg)), 0.5));
  const double a = __dadd_rn(__dmul_rn(s1, s1), __dmul_rn(__dmul_rn(ci, cj), __dmul_rn(s2, s2)));
  const double r = __dsqrt_rn(a);
  return __dmul_rn(two_r, asin(r > 1.0 ? 1.0 : r));  // a NaN stays NaN, as in the definition
}

// The definition in float64: distance, then rint(d / speed * 60). cos64: the staged
// cosines of the latitudes (Haversine, small instances) or NULL.
__device__ __forceinline__ double minutes64(const MParams& P, const double* c, const double* cos64, int i, int j,
                                            int t) {
  const double xi = c[2 * i], yi = c[2 * i + 1], xj = c[2 * j], yj = c[2 * j + 1];
  double d;
  if (P.metric == ASCHED_METRIC_HAVERSINE) {
    const double ci = cos64 ? cos64[i] : cos(__dmul_rn(xi, P.deg));
    const double cj = cos64 ? cos64[j] : cos(__dmul_rn(xj, P.deg));
    d = haversine(xi, yi, xj, yj, ci, cj, P.two_r, P.deg);
  } else {
    d = euclid(xi, yi, xj, yj);
  }
  return rint(__dmul_rn(__ddiv_rn(d, P.speed[t]), 60.0));
}

__device__ __forceinline__ int32_t checked(double m, int& bad) {
  const bool ok = m >= 0.0 && m <= 2147483647.0;  // false for NaN too
  bad |= !ok;
  return ok ? static_cast<int32_t>(m) : 0;
}

// One float32 time t32 >= 0 (or NaN): its integer in v, and whether that integer is
// certain, i.e. t32 < 2^22 lies farther than tol = rel t32 + c from every half minute.
__device__ __forceinline__ bool round_screened(float t32, float rel, float c, int32_t& v) {
  const float s = __fadd_rn(t32, 12582912.0f);  // 1.5 * 2^23: rounds t32 half to even
  const float gap = __fsub_rn(0.5f, fabsf(__fsub_rn(t32, __fsub_rn(s, 12582912.0f))));
  v = __float_as_int(s) - 0x4B400000;
  return t32 < 4194304.0f && gap > __fmaf_rn(rel, t32, c);
}

// The same where t32 < 2^22 is known or rel is infinite (every comparison then fails).
__device__ __forceinline__ bool round_screened_bounded(float t32, float rel, float c, int32_t& v) {
  const float s = __fadd_rn(t32, 12582912.0f);
  const float gap = __fsub_rn(0.5f, fabsf(__fsub_rn(t32, __fsub_rn(s, 12582912.0f))));
  v = __float_as_int(s) - 0x4B400000;
  return gap > __fmaf_rn(rel, t32, c);
}

// Drain a warp's queue of deferred entries into the output rows: each lane takes entries
// and writes the float64 result.
__device__ __forceinline__ void drain(const MParams& P, const double* c, int32_t* base, int L, int64_t LL,
                                      const int* q, int n, int lane, int& bad) {
  __syncwarp();
  for (int k = lane; k < n; k += 32) {
    const int e = q[k];
    const int i = e >> 12, j = (e >> 1) & 2047, t = e & 1;
    base[t * LL + static_cast<int64_t>(i) * L + j] = checked(minutes64(P, c, nullptr, i, j, t), bad);
  }
  __syncwarp();
}

// One deferred entry of a small instance: the pair (i, j), i <= j, of type t goes to both
// of its places in the shared-memory matrix.
__device__ __forceinline__ void resolve_small(const MParams& P, const double* c, const double* cos64, int32_t* o,
                                              int L, int e, int& bad) {
  const int i = e >> 12, j = (e >> 1) & 2047, t = e & 1;
  const int32_t v = checked(minutes64(P, c, cos64, i, j, t), bad);
  o[t * L * L + i * L + j] = v;
  o[t * L * L + j * L + i] = v;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Queue the lanes whose entry of type t is not certain in the CTA's queue (warp-uniform
// call); an entry past the queue's capacity is computed here.
__device__ __forceinline__ void enqueue(bool mine, int i, int j, int t, int* cq, unsigned& s_qn, int lane,
                                        const MParams& P, const double* c, const double* cos64, int32_t* o, int L,
                                        int& bad) {
  const unsigned m = __ballot_sync(0xffffffffu, mine);
  if (!m) return;
  const int leader = __ffs(m) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(&s_qn, static_cast<unsigned>(__popc(m)));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (!mine) return;
  const unsigned pos = base + __popc(m & ((1u << lane) - 1u));
  const int e = (i << 12) | (j << 1) | t;
  if (pos < kSmallQueue)
    cq[pos] = e;
  else
    resolve_small(P, c, cos64, o, L, e, bad);
}

// Small instances, each built whole in shared memory and written out by one bulk copy.
// The instance's scalars (S and the queue's length) alternate between two slots, so that
// thread 0 can clear the next instance's while this one's are read. Every evaluated pair
// stores its float32 results; the float64 drain after the queue barrier overwrites the
// uncertain ones. NT: the number of vehicle types.
template <bool HAV, int NT>
__global__ void __launch_bounds__(kSmallThreads, 8) travel_small_kernel(const __grid_constant__ MParams P) {
  __shared__ __align__(16) SmallStage st;
  __shared__ int cq[kSmallQueue];
  __shared__ unsigned s_mag[2], s_qn[2];
  const int lane = threadIdx.x & 31;
  const int nt = NT;
  const float k0 = P.k32[0], k1 = P.k32[1];
  const float two_r32 = static_cast<float>(P.two_r);
  int bad = 0;
  if (threadIdx.x < 2) s_mag[threadIdx.x] = s_qn[threadIdx.x] = 0u;
  __syncthreads();
  int par = 0;
  for (int b = blockIdx.x; b < P.B; b += gridDim.x) {
    const int lo = P.loc_off[b];
    const int L = P.loc_off[b + 1] - lo;
    if (!is_small(L, nt)) continue;
    const double* c = P.coords + 2 * static_cast<int64_t>(lo);
    int32_t* dst = P.travel + P.travel_off[b];
    // Every thread is past the previous instance's last barrier: its reads of the stage and
    // of its slots are done.
    if (threadIdx.x == 0) s_mag[par ^ 1] = s_qn[par ^ 1] = 0u;
    {
      const int l = threadIdx.x;  // L <= kSmallLoc <= kSmallThreads
      unsigned m = 0u;
      if (l < L) {
        double x = c[2 * l], y = c[2 * l + 1];
        if (HAV) {
          x *= P.deg;
          y *= P.deg;
        }
        const float xh = static_cast<float>(x), yh = static_cast<float>(y);
        if (HAV) {
          const double cx = cos(x);
          st.cos64[l] = cx;
          st.cphi[l] = static_cast<float>(cx);
          st.hl[l] = make_float4(xh, yh, static_cast<float>(x - static_cast<double>(xh)),
                                 static_cast<float>(y - static_cast<double>(yh)));
        } else {
          st.hl[l] = make_float4(xh, yh, 0.0f, 0.0f);
          m = __float_as_uint(fabsf(xh) + fabsf(yh));  // NaN's bits exceed every finite value
        }
      }
      if (!HAV) {
        m = __reduce_max_sync(0xffffffffu, m);
        if (lane == 0 && m) atomicMax(&s_mag[par], m);
      }
    }
    if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // the last copy has read out
    __syncthreads();
    const int phase = static_cast<int>((reinterpret_cast<uintptr_t>(dst) >> 2) & 3u);
    int32_t* o = st.out + phase;  // o[w] is dst[w]; both 16-byte aligned at the same w
    const int LL = L * L;
    float c0, c1;  // the absolute part of each type's tolerance
    float rel = P.rel_hav;
    if (!HAV) {
      const float S = __uint_as_float(s_mag[par]);
      const float magk = 9.536743e-7f * S;  // 2^-20 S
      c0 = k0 * magk + 1e-6f;
      c1 = k1 * magk + 1e-6f;
      // every time is below 2 S k (1 + 10 2^-24); false for a NaN or infinite S
      rel = 2.0f * S * fmaxf(k0, NT > 1 ? k1 : 0.0f) * 1.001f < 4194304.0f ? 2e-6f : __int_as_float(0x7f800000);
    }
    // Pair p = f (L + 1) + k: row f from column f (k < L - f), else row L - 1 - f from column k - 1.
    const int L1 = L + 1, E = L * L1 / 2;
    int f = threadIdx.x / L1, k = threadIdx.x - f * L1;
    const int df = kSmallThreads / L1, dk = kSmallThreads - df * L1;
    for (int p0 = 0; p0 < E; p0 += kSmallThreads) {
      const bool live = p0 + static_cast<int>(threadIdx.x) < E;
      int i = f, j = f + k;
      if (k >= L - f) {
        i = L - 1 - f;
        j = k - 1;
      }
      if (!live) i = j = 0;
      f += df;
      k += dk;
      if (k >= L1) {
        k -= L1;
        ++f;
      }
      const float4 a = st.hl[i], bb = st.hl[j];
      float d32;
      bool screen = true;
      if (HAV) {
        const float dx = __fadd_rn(__fsub_rn(a.x, bb.x), __fsub_rn(a.z, bb.z));
        const float dy = __fadd_rn(__fsub_rn(a.y, bb.y), __fsub_rn(a.w, bb.w));
        const float s1 = sinf(__fmul_rn(dx, 0.5f)), s2 = sinf(__fmul_rn(dy, 0.5f));
        const float h = __fadd_rn(__fmul_rn(s1, s1), __fmul_rn(__fmul_rn(st.cphi[i], st.cphi[j]), __fmul_rn(s2, s2)));
        const float r = __fsqrt_rn(h);
        screen = r <= 0.9f;
        d32 = __fmul_rn(two_r32, asinf(r));
        const float magk = two_r32 * 9.094947e-13f *  // 2 r 2^-40 (sum of |angles|)
                           (fabsf(a.x) + fabsf(bb.x) + fabsf(a.y) + fabsf(bb.y));
        c0 = k0 * magk + 1e-5f;
        c1 = k1 * magk + 1e-5f;
      } else {
        const float dx = __fsub_rn(a.x, bb.x), dy = __fsub_rn(a.y, bb.y);
        const float q = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        d32 = q > 0.0f ? __fmul_rn(q, rsqrtf(q)) : q;  // sqrt(0) = 0 exactly; NaN stays NaN
      }
      if (!live) d32 = 0.0f;  // so that its stores write the 0 of entry (0, 0), whatever the coordinates
      int32_t v0, v1 = 0;
      const bool sure0 = round_screened_bounded(__fmul_rn(d32, k0), rel, c0, v0) && screen;
      const bool sure1 = NT < 2 || (round_screened_bounded(__fmul_rn(d32, k1), rel, c1, v1) && screen);
      o[i * L + j] = v0;
      o[j * L + i] = v0;
      if (NT > 1) {
        o[LL + i * L + j] = v1;
        o[LL + j * L + i] = v1;
      }
      if (__ballot_sync(0xffffffffu, live && !(sure0 && sure1))) {  // rare: float64 for these
        enqueue(live && !sure0, i, j, 0, cq, s_qn[par], lane, P, c, st.cos64, o, L, bad);
        if (NT > 1) enqueue(live && !sure1, i, j, 1, cq, s_qn[par], lane, P, c, st.cos64, o, L, bad);
      }
    }
    __syncthreads();  // the queue is complete
    const int nq = min(static_cast<int>(s_qn[par]), kSmallQueue);
    for (int e = threadIdx.x; e < nq; e += kSmallThreads) resolve_small(P, c, st.cos64, o, L, cq[e], bad);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the writes above, before the bulk copy reads them
    __syncthreads();
    const int W = nt * LL;
    const int head = min((4 - phase) & 3, W);
    const int mid = (W - head) & ~3;
    if (threadIdx.x == 0 && mid > 0) {
      asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst + head),
                   "r"(smem_addr(o + head)), "r"(static_cast<uint32_t>(mid) * 4u)
                   : "memory");
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
    if (threadIdx.x < head) dst[threadIdx.x] = o[threadIdx.x];
    const int w = head + mid + static_cast<int>(threadIdx.x);
    if (w < W) dst[w] = o[w];
    par ^= 1;
  }
  if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // the last bulk copy is complete
  if (bad && P.status) atomicExch(P.status, ASCHED_E_INVALID);
}

// Instances that are not small: warps take rows, lanes take columns.
template <bool HAV>
__global__ void __launch_bounds__(kThreads, 4) travel_kernel(const __grid_constant__ MParams P) {
  __shared__ Stage st;
  __shared__ int queue[kWarps][kQueue];
  __shared__ unsigned s_mag;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float two_r32 = static_cast<float>(P.two_r);
  const float k0 = P.k32[0], k1 = P.k32[1];
  const int nt = P.nt;
  int bad = 0;
  for (int b = blockIdx.x; b < P.B; b += gridDim.x) {
    const int lo = P.loc_off[b];
    const int L = P.loc_off[b + 1] - lo;
    if (is_small(L, nt)) continue;
    const double* c = P.coords + 2 * static_cast<int64_t>(lo);
    int32_t* base = P.travel + P.travel_off[b];
    const int64_t LL = static_cast<int64_t>(L) * L;
    if (L > kStageLocations) {  // float64 only
      for (int i = warp; i < L; i += kWarps)
        for (int j = lane; j < L; j += 32)
          for (int t = 0; t < P.nt; ++t)
            base[t * LL + static_cast<int64_t>(i) * L + j] = checked(minutes64(P, c, nullptr, i, j, t), bad);
      continue;
    }
    __syncthreads();  // the previous instance's stage is no longer read
    if (threadIdx.x == 0) s_mag = 0u;
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
      double x = c[2 * l], y = c[2 * l + 1];
      const float xh = static_cast<float>(HAV ? x * P.deg : x), yh = static_cast<float>(HAV ? y * P.deg : y);
      st.xh[l] = xh;
      st.yh[l] = yh;
      if (HAV) {
        x *= P.deg;
        y *= P.deg;
        st.cphi[l] = static_cast<float>(cos(x));
        st.xl[l] = static_cast<float>(x - static_cast<double>(xh));
        st.yl[l] = static_cast<float>(y - static_cast<double>(yh));
      } else {
        const float m = fabsf(xh) + fabsf(yh);  // >= 0 (or NaN, whose bits exceed every finite value)
        atomicMax(&s_mag, __float_as_uint(m));
      }
    }
    __syncthreads();
    const float S = __uint_as_float(s_mag);
    int* q = queue[warp];
    int n = 0;  // queued entries (warp-uniform)
    for (int i = warp; i < L; i += kWarps) {
      int32_t* row = base + static_cast<int64_t>(i) * L;
      int32_t* row1 = row + LL;  // the same row of the second type's matrix
      for (int j0 = 0; j0 < L; j0 += 32) {
        const int j = j0 + lane;
        const bool live = j < L;
        const int jj = live ? j : i;
        float d32, rel, abs_part, magk;
        bool screen = true;
        if (HAV) {
          const float dx = __fadd_rn(__fsub_rn(st.xh[i], st.xh[jj]), __fsub_rn(st.xl[i], st.xl[jj]));
          const float dy = __fadd_rn(__fsub_rn(st.yh[i], st.yh[jj]), __fsub_rn(st.yl[i], st.yl[jj]));
          const float s1 = sinf(__fmul_rn(dx, 0.5f)), s2 = sinf(__fmul_rn(dy, 0.5f));
          const float a = __fadd_rn(__fmul_rn(s1, s1), __fmul_rn(__fmul_rn(st.cphi[i], st.cphi[jj]), __fmul_rn(s2, s2)));
          const float r = __fsqrt_rn(a);
          screen = r <= 0.9f;
          d32 = __fmul_rn(two_r32, asinf(r));
          rel = 8e-6f;
          abs_part = 1e-5f;
          magk = two_r32 * 9.094947e-13f *  // 2 r 2^-40 (sum of |angles|)
                 (fabsf(st.xh[i]) + fabsf(st.xh[jj]) + fabsf(st.yh[i]) + fabsf(st.yh[jj]));
        } else {
          const float dx = __fsub_rn(st.xh[i], st.xh[jj]), dy = __fsub_rn(st.yh[i], st.yh[jj]);
          d32 = __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)));
          rel = 2e-6f;
          abs_part = 1e-6f;
          magk = 9.536743e-7f * S;  // 2^-20 S
        }
        // One entry of type t: rounded in float32 when sure, else queued for float64.
        auto emit = [&](int t, float kt, int32_t* rowt) {
          int32_t v;
          const bool sure = round_screened(__fmul_rn(d32, kt), rel, kt * magk + abs_part, v) && screen;
          if (live && sure) rowt[j] = v;
          const unsigned need = __ballot_sync(0xffffffffu, live && !sure);
          if (need) {
            if (n + 32 > kQueue) {
              drain(P, c, base, L, LL, q, n, lane, bad);
              n = 0;
            }
            if (live && !sure) q[n + __popc(need & ((1u << lane) - 1u))] = (i << 12) | (j << 1) | t;
            n += __popc(need);
          }
        };
        emit(0, k0, row);
        if (nt > 1) emit(1, k1, row1);
      }
    }
    drain(P, c, base, L, LL, q, n, lane, bad);
  }
  if (bad && P.status) atomicExch(P.status, ASCHED_E_INVALID);
}

}  // namespace

extern "C" int asched_travel_matrix(const asched_travel_spec* spec, int32_t* travel, int32_t* status,
                                    void* stream) {
  const asched_nvtx::Range nvtx_range("asched_travel_matrix");
  if (!spec || !travel) return ASCHED_E_INVALID;
  const int B = spec->n_instances;
  if (B < 0 || spec->n_types < 1 || spec->n_types > 2) return ASCHED_E_INVALID;
  if (spec->metric != ASCHED_METRIC_EUCLIDEAN && spec->metric != ASCHED_METRIC_HAVERSINE) return ASCHED_E_INVALID;
  for (int t = 0; t < spec->n_types; ++t)
    if (!(spec->speed_kmh[t] > 0.0) || !isfinite(spec->speed_kmh[t])) return ASCHED_E_INVALID;
  if (spec->metric == ASCHED_METRIC_HAVERSINE && !(spec->radius_km >= 0.0 && isfinite(spec->radius_km)))
    return ASCHED_E_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (status && cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) {
    (void)cudaGetLastError();
    return ASCHED_E_CUDA;
  }
  if (B == 0) return ASCHED_OK;
  if (!spec->h_loc_off || !spec->loc_off || !spec->travel_off || !spec->coords) return ASCHED_E_INVALID;
  if (spec->h_loc_off[0] != 0) return ASCHED_E_INVALID;
  for (int b = 0; b < B; ++b)
    if (spec->h_loc_off[b + 1] - spec->h_loc_off[b] < 1) return ASCHED_E_INVALID;
  MParams q = {};
  q.B = B;
  q.nt = spec->n_types;
  q.metric = spec->metric;
  q.speed[0] = spec->speed_kmh[0];
  q.speed[1] = spec->n_types > 1 ? spec->speed_kmh[1] : 1.0;
  q.k32[0] = static_cast<float>(60.0 / q.speed[0]);
  q.k32[1] = static_cast<float>(60.0 / q.speed[1]);
  const double r = spec->radius_km > 0.0 ? spec->radius_km : 6371.0;
  q.two_r = 2.0 * r;
  {  // every Haversine time is at most pi r 60 / speed (a float32 margin of 2^-10)
    const double kmax = 60.0 / (q.nt > 1 && q.speed[1] < q.speed[0] ? q.speed[1] : q.speed[0]);
    q.rel_hav = 3.141592653589793 * r * kmax * (1.0 + 1.0 / 1024.0) < 4194304.0 ? 8e-6f : INFINITY;
  }
  q.deg = 3.141592653589793 / 180.0;
  q.loc_off = spec->loc_off;
  q.travel_off = spec->travel_off;
  q.coords = spec->coords;
  q.travel = travel;
  q.status = status;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return ASCHED_E_CUDA;
  }
  int64_t n_small = 0;
  for (int b = 0; b < B; ++b) n_small += is_small(spec->h_loc_off[b + 1] - spec->h_loc_off[b], q.nt);
  const bool hav = q.metric == ASCHED_METRIC_HAVERSINE;
  if (n_small > 0) {
    void (*const kernels[2][2])(MParams) = {{travel_small_kernel<false, 1>, travel_small_kernel<false, 2>},
                                            {travel_small_kernel<true, 1>, travel_small_kernel<true, 2>}};
    void (*const kern)(MParams) = kernels[hav][q.nt - 1];
    // eight 28 KB CTAs per SM want the largest shared-memory carveout (a per-device
    // attribute of the function, so it is set on every call: a host call, no device work)
    if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
        cudaSuccess) {
      (void)cudaGetLastError();
      return ASCHED_E_CUDA;
    }
    const int64_t cap = static_cast<int64_t>(sms) * 8;  // 8 CTAs of 128 threads per SM
    const int grid = static_cast<int>(n_small < cap ? n_small : cap);
    kern<<<grid, kSmallThreads, 0, st>>>(q);
    if (cudaGetLastError() != cudaSuccess) return ASCHED_E_CUDA;
  }
  if (n_small < B) {
    const int64_t cap = static_cast<int64_t>(sms) * 4;  // 4 CTAs of 256 threads per SM
    const int grid = static_cast<int>(B - n_small < cap ? B - n_small : cap);
    if (hav)
      travel_kernel<true><<<grid, kThreads, 0, st>>>(q);
    else
      travel_kernel<false><<<grid, kThreads, 0, st>>>(q);
    if (cudaGetLastError() != cudaSuccess) return ASCHED_E_CUDA;
  }
  return ASCHED_OK;
}
