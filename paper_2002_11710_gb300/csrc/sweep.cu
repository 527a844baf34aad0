// The paper's per-mission sweeps on GB300: Algorithm 2 (Neighbourhood Search,
// Section 4.2) and Algorithm 3 as printed (Section 4.3), started from the greedy
// schedule of Algorithm 1 (Section 4.1), for a batch of instances.
//
// One CTA per instance; the whole state sits in shared memory:
//   nxt/prv   doubly linked routes over nodes 0..M-1 (missions) and M+v (a sentinel
//             that is both the start and the end of vehicle v's route);
//   pos       index of a node in its route (the sentinel holds n_v, the append point);
//   veh, fl, nlen   vehicle of each mission, flight minutes and length of each route.
// Travel times come from global memory through the read-only cache.
//
// One step tries one mission j of the vehicle i whose turn it is. Its candidates are
// the nodes y on every other vehicle k: "insert j immediately before y" is insertion
// point q = pos[y] of k. The paper's parallel form gives each base a thread; here the
// candidates (about M + V of them) are spread over the block's threads. A first pass
// finds, per vehicle, the first infeasible insertion point (shared-memory atomicMin),
// which ends that vehicle's scan; a second pass takes the least (delta, k, q) of the
// points before it. The thread that evaluated the winner applies it, since only it
// knows y. Removal from i is the same for every candidate, so every thread computes it
// and every branch on it stays uniform across the block.
#include <cuda_runtime.h>
#include <stdint.h>

#include "asched.h"
#include "nvtx_range.h"

namespace {

constexpr int kMaxMissions = 4095;
constexpr int kMaxVehicles = 1024;
constexpr int kMaxNodes = 8192;
constexpr int kMaxThreads = 512;
constexpr int kIdShift = 13;
constexpr uint64_t kNoKey = ~0ull;
constexpr int kNoPos = 0x7FFFFFFF;

struct SwParams {
  int32_t B, nt, tenure, max_sweeps, lambda, accept_worse, repair, trace_cap;
  const int32_t* vehicle_order;  // at veh_off[b], or NULL
  const int32_t* mission_rank;   // at mis_off[b], or NULL
  const int32_t* loc_off;
  const int32_t* veh_off;
  const int32_t* mis_off;
  const int64_t* travel_off;
  const int32_t* travel;
  const int32_t* veh_base;
  const int32_t* veh_type;
  const int32_t* pickup;
  const int32_t* delivery;
  const int32_t* heli_only;
  const int32_t* deadline;
  const int32_t* duty_cap;
  const int32_t* horizon;
  int32_t* out_off;
  int32_t* out_route;
  int32_t* out_flight;
  int32_t* out_over;
  int32_t* info;
  uint32_t* trace_move;
  int32_t* trace_z;
};

// Shared-memory words one instance needs.
__host__ __device__ inline int sweep_words(int M, int V, int nt, bool tabu) {
  const int N = M + V;
  return 6 * N + (6 + nt) * M + 6 * V + (tabu ? M * V : 0);
}

__device__ __forceinline__ int pos0(int x) { return x > 0 ? x : 0; }

// (delta, k, q) as one unsigned key: delta's sign bit flipped so unsigned order is
// signed order, then k (10 bits) and q (13 bits).
__device__ __forceinline__ uint64_t cand_key(int d, int k, int q) {
  return (static_cast<uint64_t>(static_cast<uint32_t>(d) ^ 0x80000000u) << 32) |
         (static_cast<uint32_t>(k) << kIdShift) | static_cast<uint32_t>(q);
}
__device__ __forceinline__ int key_delta(uint64_t key) {
  return static_cast<int>(static_cast<uint32_t>(key >> 32) ^ 0x80000000u);
}

// The block's barrier: a warp barrier when the block is one warp (W).
template <bool W>
__device__ __forceinline__ void bar() {
  if (W)
    __syncwarp();
  else
    __syncthreads();
}

// Least key over the block; every thread gets it. Contains one barrier, so a caller
// must separate two calls by another barrier (red is reused).
template <bool W>
__device__ __forceinline__ uint64_t block_min(uint64_t key, uint64_t* red) {
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t other = __shfl_xor_sync(0xffffffffu, key, o);
    key = other < key ? other : key;
  }
  if (W) {
    __syncwarp();
    return key;
  }
  const int nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = key;
  __syncthreads();
  uint64_t best = red[0];
  for (int w = 1; w < nw; ++w) best = red[w] < best ? red[w] : best;
  return best;
}

struct Sw {
  // instance
  int L, V, M, N, cap, horizon, lam;
  const int32_t* T;  // [nt][L][L]
  // shared memory
  int32_t *nxt, *prv, *pos, *bnx, *sloc, *eloc;  // [N]
  int32_t *veh, *wm, *heli, *own;                // [M], own [nt][M]
  int32_t *vty, *fl, *nlen, *fbad, *scratch;     // [V]
  int32_t *vord, *mrk, *turn, *sorted;           // vehicle order [V]; mission ranks, turn lists [M]
  bool ranked;                                   // a turn's missions go by rank, not route order
  int32_t* tabu;                                 // [M][V]
};

__device__ __forceinline__ int tt(const Sw& s, int ty, int a, int b) {
  return __ldg(s.T + (static_cast<int64_t>(ty) * s.L + a) * s.L + b);
}

// Progress of a search: its step counter, objective, best so far and trace.
struct Run {
  int step, z, z_best, best_step, moves, tenure, accept_worse, trace_cap;
  bool keep_best;  // copy the links of every new best schedule into bnx
  uint32_t* trace_move;
  int32_t* trace_z;
};

// One step: mission j of vehicle i (candidates, break rule, tabu list and acceptance as
// in asched.h). Every thread calls it with the same arguments (it holds barriers);
// returns the node after j before the step, which is still on i.
template <bool PEN, bool DL, bool TABU, bool W>
__device__ __forceinline__ int sweep_step(const Sw& s, int i, int j, Run& r, uint64_t* red, bool& applied) {
  const int M = s.M, V = s.V, N = s.N, cap = s.cap, lam = s.lam;
  const int tid = threadIdx.x, nthr = blockDim.x;
  // Removal of j from i: identical for every candidate.
  const int u = s.prv[j], x = s.nxt[j];
  const int tyi = s.vty[i], fli = s.fl[i];
  const int pj = s.sloc[j], dj = s.eloc[j], wj = s.wm[j];
  int fi2 = 0;
  bool rem_ok = true;
  if (s.nlen[i] > 1) {
    const int eu = s.eloc[u], sx = s.sloc[x];
    const int link = tt(s, tyi, eu, sx);
    fi2 = fli - (tt(s, tyi, eu, pj) + s.own[tyi * M + j] + tt(s, tyi, dj, sx) - link);
    if (DL) {
      const int dep = u < M ? s.wm[u] : 0;
      rem_ok = x < M ? dep + link + s.own[tyi * M + x] <= s.wm[x] : dep + link <= s.horizon;
    }
    if (!PEN) rem_ok = rem_ok && fi2 <= cap;
  }
  const int di = fi2 - fli + (PEN ? lam * (pos0(fi2 - cap) - pos0(fli - cap)) : 0);
  const bool heli_j = s.heli[j] != 0;
  uint64_t best = kNoKey;
  int my_y = -1, my_ins = 0;
  if (rem_ok) {
    // Insert j before y (on vehicle k, point q): false if y is not a candidate; else
    // ins (the change of k's flight), feasibility, and the key when feasible.
    auto cand = [&](int y, int& k, int& q, int& ins, bool& ok, uint64_t& key) -> bool {
      k = y < M ? s.veh[y] : y - M;
      if (k == i || k < 0) return false;  // k < 0: a mission Algorithm 1 has not placed yet
      const int tyk = s.vty[k];
      if (heli_j && tyk != 0) return false;
      if (TABU && s.tabu[j * V + k] >= r.step) return false;
      q = s.pos[y];
      const int uy = s.prv[y];
      const int eu = s.eloc[uy], sy = s.sloc[y];
      const int a = tt(s, tyk, eu, pj) + s.own[tyk * M + j];
      const int bq = tt(s, tyk, dj, sy);
      ins = a + bq - (s.nlen[k] == 0 ? 0 : tt(s, tyk, eu, sy));
      const int flk = s.fl[k];
      ok = true;
      if (DL) {
        ok = (uy < M ? s.wm[uy] : 0) + a <= wj;
        ok = ok && (y < M ? wj + bq + s.own[tyk * M + y] <= s.wm[y] : wj + bq <= s.horizon);
      }
      if (!PEN) ok = ok && flk + ins <= cap;
      const int d = di + ins + (PEN ? lam * (pos0(flk + ins - cap) - pos0(flk - cap)) : 0);
      key = cand_key(d, k, q);
      return true;
    };
    // Pass 1: every candidate is evaluated once; an infeasible one marks the first
    // infeasible insertion point of its vehicle. A thread keeps the keys of its first two
    // candidates; further ones (more than 2 x threads nodes) are evaluated again in pass 2.
    uint64_t kk[2];
    int ky[2], kins[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int y = tid + c * nthr;
      kk[c] = kNoKey;
      ky[c] = y;
      kins[c] = 0;
      int k, q, ins;
      bool ok;
      uint64_t key;
      if (y < N && cand(y, k, q, ins, ok, key)) {
        if (ok) {
          kk[c] = key;
          kins[c] = ins;
        } else {
          atomicMin(&s.fbad[k], q);
        }
      }
    }
    for (int y = tid + 2 * nthr; y < N; y += nthr) {
      int k, q, ins;
      bool ok;
      uint64_t key;
      if (cand(y, k, q, ins, ok, key) && !ok) atomicMin(&s.fbad[k], q);
    }
    bar<W>();
    // Pass 2: the least (delta, k, q) before each vehicle's first infeasible point.
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const uint64_t key = kk[c];
      if (key == kNoKey) continue;
      const int k = static_cast<int>((key >> kIdShift) & 0x3FFu), q = static_cast<int>(key & 0x1FFFu);
      if (q < s.fbad[k] && key < best) {
        best = key;
        my_y = ky[c];
        my_ins = kins[c];
      }
    }
    for (int y = tid + 2 * nthr; y < N; y += nthr) {
      int k, q, ins;
      bool ok;
      uint64_t key;
      if (cand(y, k, q, ins, ok, key) && ok && q < s.fbad[k] && key < best) {
        best = key;
        my_y = y;
        my_ins = ins;
      }
    }
  }
  const uint64_t win = rem_ok ? block_min<W>(best, red) : kNoKey;
  const int d = win == kNoKey ? 0 : key_delta(win);
  const bool apply = win != kNoKey && (d < 0 || r.accept_worse);
  if (apply && best == win) {
    // remove j from i
    s.nxt[u] = x;
    s.prv[x] = u;
    for (int w = x;; w = s.nxt[w]) {
      s.pos[w] -= 1;
      if (w == M + i) break;
    }
    s.nlen[i] -= 1;
    s.fl[i] = fi2;
    // insert j before y on k
    const int k = static_cast<int>((win >> kIdShift) & 0x3FFu);
    const int uy = s.prv[my_y];
    s.nxt[uy] = j;
    s.prv[j] = uy;
    s.nxt[j] = my_y;
    s.prv[my_y] = j;
    s.pos[j] = s.pos[my_y];
    for (int w = my_y;; w = s.nxt[w]) {
      s.pos[w] += 1;
      if (w == M + k) break;
    }
    s.nlen[k] += 1;
    s.fl[k] += my_ins;
    s.veh[j] = k;
    if (TABU) s.tabu[j * V + i] = r.step + r.tenure;
    if (r.step < r.trace_cap) {
      const int64_t t = static_cast<int64_t>(blockIdx.x) * r.trace_cap + r.step;
      if (r.trace_move) r.trace_move[t] = (static_cast<uint32_t>(j) << kIdShift) | my_y;
      if (r.trace_z) r.trace_z[t] = r.z + d;
    }
  } else if (!apply && tid == 0 && r.step < r.trace_cap) {
    const int64_t t = static_cast<int64_t>(blockIdx.x) * r.trace_cap + r.step;
    if (r.trace_move) r.trace_move[t] = ASCHED_NULL_MOVE;
    if (r.trace_z) r.trace_z[t] = r.z;
  }
  for (int v = tid; v < V; v += nthr) s.fbad[v] = kNoPos;
  bool improved = false;
  if (apply) {
    r.z += d;
    ++r.moves;
    applied = true;
    if (r.z < r.z_best) {
      r.z_best = r.z;
      r.best_step = r.step;
      improved = true;
    }
  }
  bar<W>();
  if (improved && r.keep_best)
    for (int w = tid; w < N; w += nthr) s.bnx[w] = s.nxt[w];
  ++r.step;
  return x;
}

// One sweep: the vehicles' turns in the given order; a turn tries the vehicle's missions
// as its route stands when the turn starts, in route order or by increasing rank (missions
// only leave the vehicle during its turn, and are skipped once gone). Returns whether a
// move was applied.
template <bool PEN, bool DL, bool TABU, bool W>
__device__ __forceinline__ bool sweep_pass(const Sw& s, Run& r, uint64_t* red) {
  const int M = s.M, tid = threadIdx.x, nthr = blockDim.x;
  bool applied = false;
  for (int ii = 0; ii < s.V; ++ii) {
    const int i = s.vord[ii];
    const int n = s.nlen[i];
    bar<W>();  // every thread is done with the previous turn's list
    if (tid == 0) {
      int k = 0;
      for (int w = s.nxt[M + i]; w != M + i; w = s.nxt[w]) s.turn[k++] = w;
    }
    const int32_t* list = s.turn;
    if (s.ranked) {
      bar<W>();
      for (int k = tid; k < n; k += nthr) {  // place each mission at its rank among the turn's
        const int m = s.turn[k], rm = s.mrk[m];
        int at = 0;
        for (int x = 0; x < n; ++x) at += s.mrk[s.turn[x]] < rm;
        s.sorted[at] = m;
      }
      list = s.sorted;
    }
    bar<W>();
    for (int k = 0; k < n; ++k) {
      const int j = list[k];
      if (s.veh[j] == i) sweep_step<PEN, DL, TABU, W>(s, i, j, r, red, applied);
    }
  }
  return applied;
}

// Algorithm 1's choice for mission m: the least (objective increase, vehicle) among the
// vehicles it can be appended to; kNoKey when none. One thread per vehicle.
template <bool PEN, bool DL, bool W>
__device__ __forceinline__ uint64_t greedy_pick(const Sw& s, int m, uint64_t* red) {
  const int M = s.M;
  const int w = s.wm[m];
  uint64_t key = kNoKey;
  for (int v = threadIdx.x; v < s.V; v += blockDim.x) {
    const int ty = s.vty[v], bl = s.eloc[M + v];
    const int last = s.prv[M + v];
    const int a = tt(s, ty, s.eloc[last], s.sloc[m]) + s.own[ty * M + m];
    const int bret = tt(s, ty, s.eloc[m], bl);
    const int old = last == M + v ? 0 : tt(s, ty, s.eloc[last], bl);
    const int app = a + bret - old;
    const int f = s.fl[v];
    bool ok = !(s.heli[m] && ty != 0);
    if (DL) ok = ok && ((last < M ? s.wm[last] : 0) + a <= w) && (w + bret <= s.horizon);
    int score = app;
    if (PEN)
      score += s.lam * (pos0(f + app - s.cap) - pos0(f - s.cap));
    else
      ok = ok && (f + app <= s.cap);
    if (ok) {
      const uint64_t kv = cand_key(score, 0, v);
      key = kv < key ? kv : key;
    }
  }
  return block_min<W>(key, red);
}

// ONE_WARP: the 32-thread launch of small instances, bounded to 64 registers so that 32
// CTAs (the most an SM holds) are resident; otherwise up to 512 threads.
template <bool PEN, bool DL, bool TABU, bool ONE_WARP>
__global__ void __launch_bounds__(ONE_WARP ? 32 : kMaxThreads, ONE_WARP ? 32 : 1)
    sweep_kernel(const __grid_constant__ SwParams Q) {
  extern __shared__ __align__(16) int32_t g_sw[];
  __shared__ uint64_t s_red[kMaxThreads / 32];
  __shared__ int s_int[4];
  const int b = blockIdx.x;
  const int tid = threadIdx.x, nthr = blockDim.x;
  Sw s;
  const int lo = Q.loc_off[b], vo = Q.veh_off[b], mo = Q.mis_off[b];
  s.L = Q.loc_off[b + 1] - lo;
  s.V = Q.veh_off[b + 1] - vo;
  s.M = Q.mis_off[b + 1] - mo;
  s.N = s.M + s.V;
  s.cap = Q.duty_cap[b];
  s.horizon = Q.horizon[b];
  s.lam = PEN ? Q.lambda : 0;
  s.T = Q.travel + Q.travel_off[b];
  const int L = s.L, V = s.V, M = s.M, N = s.N, nt = Q.nt;
  const int32_t* vbase = Q.veh_base + vo;
  const int32_t* vtype = Q.veh_type ? Q.veh_type + vo : nullptr;
  const int32_t* pick = Q.pickup + mo;
  const int32_t* deli = Q.delivery + mo;
  const int32_t* hel = Q.heli_only ? Q.heli_only + mo : nullptr;
  const int32_t* dln = DL ? Q.deadline + mo : nullptr;
  int32_t* info = Q.info + static_cast<int64_t>(b) * ASCHED_INFO_LEN;
  int32_t* p = g_sw;
  s.nxt = p; p += N;
  s.prv = p; p += N;
  s.pos = p; p += N;
  s.bnx = p; p += N;
  s.sloc = p; p += N;
  s.eloc = p; p += N;
  s.veh = p; p += M;
  s.wm = p; p += M;
  s.heli = p; p += M;
  s.own = p; p += nt * M;
  s.vty = p; p += V;
  s.fl = p; p += V;
  s.nlen = p; p += V;
  s.fbad = p; p += V;
  s.scratch = p; p += V;
  s.vord = p; p += V;
  s.mrk = p; p += M;
  s.turn = p; p += M;
  s.sorted = p; p += M;
  s.ranked = Q.mission_rank != nullptr;
  s.tabu = p;

  // ---- load and validate (the same checks as the full-neighbourhood search)
  if (tid < 4) s_int[tid] = 0;
  __syncthreads();
  int bad = 0;
  for (int m = tid; m < M; m += nthr) {
    const int pk = pick[m], d = deli[m];
    const int h = hel ? hel[m] : 0;
    bad |= (pk < 0) | (pk >= L) | (d < 0) | (d >= L) | (pk == d) | (h < 0) | (h > 1);
    s.sloc[m] = pk;
    s.eloc[m] = d;
    s.heli[m] = h;
    s.wm[m] = DL ? dln[m] : 0;
    s.mrk[m] = Q.mission_rank ? Q.mission_rank[mo + m] : m;
  }
  for (int v = tid; v < V; v += nthr) {
    const int bl = vbase[v];
    const int ty = vtype ? vtype[v] : 0;
    bad |= (bl < 0) | (bl >= L) | (ty < 0) | (ty >= nt);
    s.sloc[M + v] = bl;
    s.eloc[M + v] = bl;
    s.vty[v] = ty;
    s.vord[v] = Q.vehicle_order ? Q.vehicle_order[vo + v] : v;
  }
  int maxT = 0;
  {  // the matrices, 16 bytes per load between an unaligned head and tail
    const int64_t n = static_cast<int64_t>(nt) * L * L;
    const int64_t head = min(static_cast<int64_t>((16u - (reinterpret_cast<uintptr_t>(s.T) & 15u)) & 15u) / 4, n);
    const int64_t n4 = (n - head) >> 2;
    auto see = [&](int t) {
      bad |= t < 0;
      maxT = t > maxT ? t : maxT;
    };
    for (int64_t x = tid; x < head; x += nthr) see(__ldg(s.T + x));
    const int4* T4 = reinterpret_cast<const int4*>(s.T + head);
    for (int64_t x = tid; x < n4; x += nthr) {
      const int4 t = __ldg(T4 + x);
      see(t.x);
      see(t.y);
      see(t.z);
      see(t.w);
    }
    for (int64_t x = head + 4 * n4 + tid; x < n; x += nthr) see(__ldg(s.T + x));
  }
  for (int o = 16; o > 0; o >>= 1) {
    const int other = __shfl_xor_sync(0xffffffffu, maxT, o);
    maxT = other > maxT ? other : maxT;
  }
  if ((tid & 31) == 0) atomicMax(&s_int[0], maxT);
  int status = __syncthreads_or(bad) ? ASCHED_E_INVALID : ASCHED_OK;
  if (status == ASCHED_OK) {
    // 2 (2M + V + 2) maxT (1 + lambda) < 2^31 keeps every int32 sum in range.
    const double bound = 2.0 * (2.0 * M + V + 2.0) * static_cast<double>(s_int[0]) *
                         (1.0 + static_cast<double>(s.lam));
    if (!(bound < 2147483648.0)) status = ASCHED_E_OVERFLOW_GUARD;
  }
  if (status == ASCHED_OK && (Q.vehicle_order || Q.mission_rank)) {
    // the orders must be permutations (fbad and turn serve as counters here)
    for (int v = tid; v < V; v += nthr) s.fbad[v] = 0;
    for (int m = tid; m < M; m += nthr) s.turn[m] = 0;
    __syncthreads();
    int badp = 0;
    for (int v = tid; v < V; v += nthr) {
      const int x = s.vord[v];
      if (x < 0 || x >= V) badp = 1;
      else atomicAdd(&s.fbad[x], 1);
    }
    for (int m = tid; m < M; m += nthr) {
      const int x = s.mrk[m];
      if (x < 0 || x >= M) badp = 1;
      else atomicAdd(&s.turn[x], 1);
    }
    __syncthreads();
    for (int v = tid; v < V; v += nthr) badp |= s.fbad[v] != 1;
    for (int m = tid; m < M; m += nthr) badp |= s.turn[m] != 1;
    if (__syncthreads_or(badp)) status = ASCHED_E_INVALID;
  }

  // ---- in-mission legs per travel layer, empty routes, tabu list
  if (status == ASCHED_OK) {
    for (int x = tid; x < nt * M; x += nthr) {
      const int t = x / M, m = x - t * M;
      s.own[x] = tt(s, t, s.sloc[m], s.eloc[m]);
    }
    for (int v = tid; v < V; v += nthr) {
      s.nxt[M + v] = M + v;
      s.prv[M + v] = M + v;
      s.fl[v] = 0;
      s.fbad[v] = kNoPos;
    }
    if (TABU)
      for (int x = tid; x < M * V; x += nthr) s.tabu[x] = -1;
  }
  __syncthreads();

  // ---- Algorithm 1: missions heli-only first, then by (deadline, id); each appended
  // to the vehicle whose objective grows least among those that stay feasible (ties to
  // the lowest index). One thread per vehicle, as in the paper's parallel form. With
  // the repair flag, a mission that fits nowhere triggers one Neighbourhood Search sweep
  // over the partial schedule and one more try (unplaced missions have veh = -1).
  if (status == ASCHED_OK) {
    int32_t* order = s.bnx;
    for (int m = tid; m < M; m += nthr) {
      const int hm = s.heli[m] ? 0 : 1, wmv = s.wm[m];
      int r = 0;
      for (int k = 0; k < M; ++k) {
        const int hk = s.heli[k] ? 0 : 1, wk = s.wm[k];
        r += (hk < hm) || (hk == hm && (wk < wmv || (wk == wmv && k < m)));
      }
      order[r] = m;
      s.veh[m] = -1;
    }
    for (int v = tid; v < V; v += nthr) {
      s.nlen[v] = 0;
      s.pos[M + v] = 0;
    }
    __syncthreads();
    int fail = 0;
    for (int r = 0; r < M; ++r) {
      const int m = order[r];
      uint64_t key = greedy_pick<PEN, DL, ONE_WARP>(s, m, s_red);
      if (key == kNoKey && Q.repair && r > 0) {
        bar<ONE_WARP>();  // s_red is read by every thread before the sweep reuses it
        Run rep = {};
        rep.keep_best = false;
        if (sweep_pass<PEN, DL, false, ONE_WARP>(s, rep, s_red)) key = greedy_pick<PEN, DL, ONE_WARP>(s, m, s_red);
      }
      if (key == kNoKey) {
        fail = 1;
        break;
      }
      if (tid == 0) {
        const int v = static_cast<int>(key & 0x1FFFu);
        const int last = s.prv[M + v];
        const int ty = s.vty[v], bl = s.eloc[M + v];
        const int a = tt(s, ty, s.eloc[last], s.sloc[m]) + s.own[ty * M + m];
        const int bret = tt(s, ty, s.eloc[m], bl);
        const int old = last == M + v ? 0 : tt(s, ty, s.eloc[last], bl);
        s.nxt[last] = m;
        s.prv[m] = last;
        s.nxt[m] = M + v;
        s.prv[M + v] = m;
        s.veh[m] = v;
        s.pos[m] = s.nlen[v];
        s.nlen[v] += 1;
        s.pos[M + v] = s.nlen[v];
        s.fl[v] += a + bret - old;
      }
      bar<ONE_WARP>();
    }
    if (fail) status = ASCHED_E_INFEASIBLE_INIT;
  }

  // ---- initial objective; the greedy schedule is the first best
  Run run = {};
  if (status == ASCHED_OK) {
    int part = 0;
    for (int v = tid; v < V; v += nthr) part += s.fl[v] + s.lam * pos0(s.fl[v] - s.cap);
    atomicAdd(&s_int[1], part);
    for (int x = tid; x < N; x += nthr) s.bnx[x] = s.nxt[x];
    __syncthreads();
    run.z = run.z_best = s_int[1];
  }
  const int z_init = run.z;
  run.best_step = -1;
  run.tenure = Q.tenure;
  run.accept_worse = Q.accept_worse;
  run.trace_cap = Q.trace_cap;
  run.trace_move = Q.trace_move;
  run.trace_z = Q.trace_z;
  run.keep_best = true;
  int sweeps = 0;

  // ---- the sweeps
  if (status == ASCHED_OK) {
    bool go_on = true;
    while (go_on && sweeps < Q.max_sweeps) {
      const int zb0 = run.z_best;
      const bool applied = sweep_pass<PEN, DL, TABU, ONE_WARP>(s, run, s_red);
      ++sweeps;
      go_on = Q.accept_worse ? (run.z_best < zb0) : applied;
    }
  }
  __syncthreads();

  // ---- best schedule out: CSR from the saved links, flight and overflow per vehicle
  if (status == ASCHED_OK) {
    for (int v = tid; v < V; v += nthr) {
      int n = 0;
      for (int w = s.bnx[M + v]; w != M + v; w = s.bnx[w]) ++n;
      s.scratch[v] = n;
    }
    __syncthreads();
    if (tid == 0) {
      int acc = 0;
      for (int v = 0; v < V; ++v) {
        const int n = s.scratch[v];
        s.scratch[v] = acc;
        acc += n;
      }
    }
    __syncthreads();
    int32_t* off = Q.out_off + vo + b;
    int32_t* route = Q.out_route + mo;
    for (int v = tid; v < V; v += nthr) {
      const int ty = s.vty[v], bl = s.eloc[M + v];
      const int k0 = s.scratch[v];
      int k = k0, f = 0, e = bl;
      off[v] = k0;
      for (int w = s.bnx[M + v]; w != M + v; w = s.bnx[w]) {
        route[k++] = w;
        f += tt(s, ty, e, s.sloc[w]) + s.own[ty * M + w];
        e = s.eloc[w];
      }
      if (k > k0) f += tt(s, ty, e, bl);  // an empty route flies nothing
      if (v == V - 1) off[V] = k;
      if (Q.out_flight) Q.out_flight[vo + v] = f;
      if (Q.out_over) Q.out_over[vo + v] = pos0(f - s.cap);
    }
  }
  if (tid == 0) {
    info[ASCHED_INFO_STATUS] = status;
    info[ASCHED_INFO_Z_BEST] = status == ASCHED_OK ? run.z_best : 0;
    info[ASCHED_INFO_BEST_IT] = status == ASCHED_OK ? run.best_step : 0;
    info[ASCHED_INFO_Z_INIT] = status == ASCHED_OK ? z_init : 0;
    info[ASCHED_INFO_Z_FINAL] = status == ASCHED_OK ? run.z : 0;
    info[ASCHED_INFO_ITERS] = sweeps;
    info[ASCHED_INFO_MOVES] = run.moves;
    info[ASCHED_INFO_STEPS] = run.step;
  }
}

template <bool PEN, bool DL, bool TABU, bool W>
void* sweep_ptr() {
  return reinterpret_cast<void*>(&sweep_kernel<PEN, DL, TABU, W>);
}

template <bool W>
void* pick_sweep_w(bool pen, bool dl, bool tabu) {
  if (pen) {
    if (dl) return tabu ? sweep_ptr<true, true, true, W>() : sweep_ptr<true, true, false, W>();
    return tabu ? sweep_ptr<true, false, true, W>() : sweep_ptr<true, false, false, W>();
  }
  if (dl) return tabu ? sweep_ptr<false, true, true, W>() : sweep_ptr<false, true, false, W>();
  return tabu ? sweep_ptr<false, false, true, W>() : sweep_ptr<false, false, false, W>();
}

void* pick_sweep(bool pen, bool dl, bool tabu, bool one_warp) {
  return one_warp ? pick_sweep_w<true>(pen, dl, tabu) : pick_sweep_w<false>(pen, dl, tabu);
}

}  // namespace

extern "C" int asched_sweep_batch(const asched_batch* bt, int32_t algorithm, const asched_params* p,
                                  const asched_sweep_orders* orders, const asched_batch_result* out,
                                  const asched_sweep_trace* trace, void* stream) {
  const asched_nvtx::Range nvtx_range("asched_sweep_batch");
  if (!bt || !p || !out) return ASCHED_E_INVALID;
  if (algorithm != ASCHED_SWEEP_NEIGHBOURHOOD && algorithm != ASCHED_SWEEP_TABU) return ASCHED_E_INVALID;
  if (p->tenure < 0 || p->iterations < 0 || p->lambda < 0) return ASCHED_E_INVALID;
  if (p->cap_mode != ASCHED_HARD && p->cap_mode != ASCHED_PENALTY) return ASCHED_E_INVALID;
  if (p->cluster_size != 0 && p->cluster_size != 1) return ASCHED_E_INVALID;
  if (p->block_threads != 0 && (p->block_threads < 32 || p->block_threads > kMaxThreads || p->block_threads % 32))
    return ASCHED_E_INVALID;
  if ((p->flags & ~(ASCHED_SWEEP_ACCEPT_WORSE | ASCHED_SWEEP_REPAIR)) != 0) return ASCHED_E_INVALID;
  const bool accept_worse = (p->flags & ASCHED_SWEEP_ACCEPT_WORSE) != 0;
  if (accept_worse && algorithm != ASCHED_SWEEP_TABU) return ASCHED_E_INVALID;
  if (trace && trace->capacity < 0) return ASCHED_E_INVALID;
  const int B = bt->n_instances;
  if (B < 0 || bt->n_types < 1 || bt->n_types > 2) return ASCHED_E_INVALID;
  if (B == 0) return ASCHED_OK;
  if (!bt->h_loc_off || !bt->h_veh_off || !bt->h_mis_off || !bt->loc_off || !bt->veh_off || !bt->mis_off ||
      !bt->travel_off || !bt->travel || !bt->veh_base || !bt->pickup || !bt->delivery || !bt->duty_cap ||
      !bt->horizon)
    return ASCHED_E_INVALID;
  if (!out->route_off || !out->route || !out->info) return ASCHED_E_INVALID;
  const bool tabu = algorithm == ASCHED_SWEEP_TABU;
  int dev = 0, limit = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return ASCHED_E_CUDA;
  }
  int max_words = 0, max_nodes = 1;
  for (int b = 0; b < B; ++b) {
    const int L = bt->h_loc_off[b + 1] - bt->h_loc_off[b];
    const int V = bt->h_veh_off[b + 1] - bt->h_veh_off[b];
    const int M = bt->h_mis_off[b + 1] - bt->h_mis_off[b];
    if (L < 1 || V < 1 || M < 0) return ASCHED_E_INVALID;
    if (V > kMaxVehicles || M > kMaxMissions || M + V > kMaxNodes) return ASCHED_E_TOO_LARGE;
    if (static_cast<int64_t>(p->iterations) * M + p->tenure >= 2147483647LL) return ASCHED_E_INVALID;
    const int w = sweep_words(M, V, bt->n_types, tabu);
    if (static_cast<int64_t>(w) * 4 > limit) return ASCHED_E_TOO_LARGE;
    max_words = w > max_words ? w : max_words;
    max_nodes = M + V > max_nodes ? M + V : max_nodes;
  }
  int threads = p->block_threads;
  if (threads == 0) threads = max_nodes <= 64 ? 32 : max_nodes <= 256 ? 64 : max_nodes <= 1024 ? 128 : 256;
  const size_t bytes = static_cast<size_t>(max_words) * 4;
  void* fn = pick_sweep(p->cap_mode == ASCHED_PENALTY, bt->deadline != nullptr, tabu, threads == 32);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    return ASCHED_E_CUDA;
  }
  SwParams q = {};
  q.B = B;
  q.nt = bt->n_types;
  q.tenure = p->tenure;
  q.max_sweeps = p->iterations;
  q.lambda = p->cap_mode == ASCHED_PENALTY ? p->lambda : 0;
  q.accept_worse = accept_worse ? 1 : 0;
  q.repair = (p->flags & ASCHED_SWEEP_REPAIR) ? 1 : 0;
  q.trace_cap = trace ? trace->capacity : 0;
  q.loc_off = bt->loc_off;
  q.veh_off = bt->veh_off;
  q.mis_off = bt->mis_off;
  q.travel_off = bt->travel_off;
  q.travel = bt->travel;
  q.veh_base = bt->veh_base;
  q.veh_type = bt->veh_type;
  q.pickup = bt->pickup;
  q.delivery = bt->delivery;
  q.heli_only = bt->heli_only;
  q.deadline = bt->deadline;
  q.duty_cap = bt->duty_cap;
  q.horizon = bt->horizon;
  q.out_off = out->route_off;
  q.out_route = out->route;
  q.out_flight = out->flight;
  q.out_over = out->overflow;
  q.info = out->info;
  q.vehicle_order = orders ? orders->vehicle_order : nullptr;
  q.mission_rank = orders ? orders->mission_rank : nullptr;
  q.trace_move = trace ? trace->move : nullptr;
  q.trace_z = trace ? trace->z : nullptr;
  void* args[] = {&q};
  if (cudaLaunchKernel(fn, dim3(B), dim3(threads), args, bytes, static_cast<cudaStream_t>(stream)) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    return ASCHED_E_CUDA;
  }
  return ASCHED_OK;
}
