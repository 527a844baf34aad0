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
//              sum of the four magnitudes, then differences, squares, sum, correctly
//              rounded square root and the product with a rounded 60 / speed add below
//              6 * 2^-24 relative; screened at 2e-6 t + (60 / speed) 2^-20 S + 1e-6, S the
//              instance's largest |x| + |y|;
//   Haversine  angles staged as float pairs hi + lo (lo = float(v - hi)), so a difference
//              (hi_i - hi_j) + (lo_i - lo_j) is within 2 * 2^-24 of itself plus 2^-47 of
//              the magnitudes; half-angle differences, sinf (2 ulp), squares, cos(phi)
//              staged from float64, sum, square root and asinf (2 ulp) with its condition
//              number below 1.9 for sqrt(a) <= 0.9 (larger values go to float64 outright)
//              add below 1.8e-6 relative; screened at 8e-6 t + (60 / speed) 2 r 2^-40
//              (sum of |angles|) + 1e-5.
// Times of 2^22 minutes or more also go to float64. The float64 path is the expression
// above, on the original float64 coordinates. Lanes that need it queue (row, column,
// type) in shared memory, and the whole warp drains its queue when it fills and at the
// end of the instance, so float64 work runs on full warps and follows the number of such
// entries.
//
// One CTA per instance (grid-stride over instances): the instance's coordinates are
// staged once in shared memory (angles in radians and cos(phi) for Haversine); warps
// take rows, lanes take columns, so a row's writes are contiguous. An instance with more
// locations than the stage holds goes through float64 alone.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "asched.h"

namespace {

constexpr int kStageLocations = 2048;  // 5 floats per location: 40 KB of shared memory
constexpr int kWarps = 8;
constexpr int kQueue = 128;  // deferred float64 entries per warp

struct MParams {
  int32_t B, nt, metric;
  double speed[2];
  float k32[2];  // float(60 / speed)
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

__device__ __forceinline__ double euclid(double xi, double yi, double xj, double yj) {
  const double dx = __dsub_rn(xi, xj), dy = __dsub_rn(yi, yj);
  return __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

__device__ __forceinline__ double haversine(double lati, double loni, double latj, double lonj, double two_r,
                                            double deg) {
  const double phi_i = __dmul_rn(lati, deg), phi_j = __dmul_rn(latj, deg);
  const double s1 = sin(__dmul_rn(__dsub_rn(phi_i, phi_j), 0.5));
  const double s2 = sin(__dmul_rn(__dsub_rn(__dmul_rn(loni, deg), __dmul_rn(lonj, deg)), 0.5));
  const double a = __dadd_rn(__dmul_rn(s1, s1), __dmul_rn(__dmul_rn(cos(phi_i), cos(phi_j)), __dmul_rn(s2, s2)));
  const double r = __dsqrt_rn(a);
  return __dmul_rn(two_r, asin(r > 1.0 ? 1.0 : r));  // a NaN stays NaN, as in the definition
}

// The definition in float64: distance, then rint(d / speed * 60).
__device__ __forceinline__ double minutes64(const MParams& P, const double* c, int i, int j, int t) {
  const double xi = c[2 * i], yi = c[2 * i + 1], xj = c[2 * j], yj = c[2 * j + 1];
  const double d = P.metric == ASCHED_METRIC_HAVERSINE ? haversine(xi, yi, xj, yj, P.two_r, P.deg)
                                                       : euclid(xi, yi, xj, yj);
  return rint(__dmul_rn(__ddiv_rn(d, P.speed[t]), 60.0));
}

__device__ __forceinline__ int32_t checked(double m, int& bad) {
  const bool ok = m >= 0.0 && m <= 2147483647.0;  // false for NaN too
  bad |= !ok;
  return ok ? static_cast<int32_t>(m) : 0;
}

// Drain a warp's queue of deferred entries: each lane takes entries and writes the
// float64 result.
__device__ __forceinline__ void drain(const MParams& P, const double* c, int32_t* base, int L, int64_t LL,
                                      const int* q, int n, int lane, int& bad) {
  __syncwarp();
  for (int k = lane; k < n; k += 32) {
    const int e = q[k];
    const int i = e >> 12, j = (e >> 1) & 2047, t = e & 1;
    base[t * LL + static_cast<int64_t>(i) * L + j] = checked(minutes64(P, c, i, j, t), bad);
  }
  __syncwarp();
}

template <bool HAV>
__global__ void __launch_bounds__(kWarps * 32) travel_kernel(const __grid_constant__ MParams P) {
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
    const double* c = P.coords + 2 * static_cast<int64_t>(lo);
    int32_t* base = P.travel + P.travel_off[b];
    const int64_t LL = static_cast<int64_t>(L) * L;
    if (L > kStageLocations) {  // float64 only
      for (int i = warp; i < L; i += kWarps)
        for (int j = lane; j < L; j += 32)
          for (int t = 0; t < P.nt; ++t) base[t * LL + static_cast<int64_t>(i) * L + j] = checked(minutes64(P, c, i, j, t), bad);
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
          const float t32 = __fmul_rn(d32, kt);
          const float tol = rel * t32 + kt * magk + abs_part;
          const float frac = t32 - floorf(t32);  // exact for 0 <= t32 < 2^22
          const bool sure = screen && t32 >= 0.0f && t32 < 4194304.0f && fabsf(frac - 0.5f) > tol;
          if (live && sure) rowt[j] = static_cast<int32_t>(rintf(t32));
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
        if (HAV) {  // (this loop, written out, measured faster here than through emit)
          for (int t = 0; t < P.nt; ++t) {
            const float t32 = __fmul_rn(d32, P.k32[t]);
            const float tol = rel * t32 + P.k32[t] * magk + abs_part;
            const float frac = t32 - floorf(t32);  // exact for 0 <= t32 < 2^22
            const bool sure = screen && t32 >= 0.0f && t32 < 4194304.0f && fabsf(frac - 0.5f) > tol;
            if (live && sure) row[t * LL + j] = static_cast<int32_t>(rintf(t32));
            const unsigned need = __ballot_sync(0xffffffffu, live && !sure);
            if (need) {
              if (n + 32 > kQueue) {
                drain(P, c, base, L, LL, q, n, lane, bad);
                n = 0;
              }
              if (live && !sure) q[n + __popc(need & ((1u << lane) - 1u))] = (i << 12) | (j << 1) | t;
              n += __popc(need);
            }
          }
        } else {  // constant indices keep both types' constants in registers
          emit(0, k0, row);
          if (nt > 1) emit(1, k1, row1);
        }
      }
    }
    drain(P, c, base, L, LL, q, n, lane, bad);
  }
  if (bad && P.status) atomicExch(P.status, ASCHED_E_INVALID);
}

}  // namespace

extern "C" int asched_travel_matrix(const asched_travel_spec* spec, int32_t* travel, int32_t* status,
                                    void* stream) {
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
  const int64_t cap = static_cast<int64_t>(sms) * 4;  // up to 4 CTAs of 256 threads per SM
  const int grid = static_cast<int>(B < cap ? B : cap);
  if (q.metric == ASCHED_METRIC_HAVERSINE)
    travel_kernel<true><<<grid, kWarps * 32, 0, st>>>(q);
  else
    travel_kernel<false><<<grid, kWarps * 32, 0, st>>>(q);
  if (cudaGetLastError() != cudaSuccess) return ASCHED_E_CUDA;
  return ASCHED_OK;
}
