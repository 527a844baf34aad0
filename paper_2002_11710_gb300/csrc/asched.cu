// asched.cu - GB300 (sm_103a) Tabu search for air-ambulance fleet scheduling.
//
// Method: Tassone & Choudhury, "Algorithms for Optimizing Fleet Scheduling of Air
// Ambulances" (arXiv 2002.11710): model of Section 3 (obj_s, con1-con13), greedy
// start of Algorithm 1 (Section 4.1), Tabu search of Algorithm 3 (Section 4.3)
// widened to the whole relocate + swap neighbourhood every iteration. The readings
// of the paper that fix the move set, move ids, tabu attribute, aspiration and
// tie-break are stated in include/asched.h.
//
// Design (one instance per launch):
//   * One persistent launch runs every iteration. The grid is one thread-block
//     cluster of C CTAs (C = 1..16), or K such clusters for large neighbourhoods, one
//     CTA per SM. Each CTA holds a complete copy of the instance and of the search
//     state in shared memory and applies every move itself, so the only traffic
//     between CTAs per iteration is one 64-bit key per CTA: a relaxed DSMEM store of a
//     key tagged with the iteration inside a cluster, and a relaxed global store of the
//     cluster's key between clusters, each polled by the receivers with a bounded wait.
//   * Shared memory holds two node-by-mission gather tables built once per launch:
//       A[t][l][m] = T_t[l][p_m] + T_t[p_m][d_m]   (fly from location l to m's pickup, then m)
//       B[t][l][m] = T_t[d_m][l]                   (from m's delivery to location l)
//     with the mission index innermost and rows padded to a multiple of 32 words,
//     so that 32 lanes reading 32 consecutive missions of any row hit 32 banks; or,
//     for instances whose tables do not fit, the travel matrix itself in int16.
//   * The schedule is a doubly linked list over nodes (missions 0..M-1 and route
//     ends M..M+V-1), with per-node records (removal delta, gap leg, slot cost,
//     table row offsets, cap slack, deadline slacks) in an SoA. A node's records
//     depend only on its own links, vehicle and route flight and on static tables, so
//     applying a move rewrites them in place, in one pass (one thread per node) after
//     one barrier that follows the decode: only the nodes of the one or two routes
//     the move changes are recomputed; the rest are current.
//   * Every move (relocate (m, y) and swap (a, b)) is evaluated in O(1) from the
//     records and the tables; the per-thread, warp (redux.sync), CTA (shared
//     memory), cluster (DSMEM) and grid (L2) minimum of the key
//     ((delta ^ 2^31) << 32) | id is independent of how moves are split over threads,
//     so any launch shape gives the same trajectory.
//   * The tabu list is a V x M table of iteration stamps in shared memory.
//   * The batch and serving kernels run the same search per instance, one CTA or one
//     cluster each, with one more record per mission (a relocation's source-route
//     delta), relocation items of four missions and the pass over every pair of
//     missions in its short form, the swaps of route neighbours in a pass of their own.

#include <cuda_runtime.h>
#include <stdint.h>

#include "asched.h"
#include "nvtx_range.h"

namespace {

constexpr uint32_t kSwapBit = 0x80000000u;
constexpr uint32_t kNullMove = 0xFFFFFFFFu;
constexpr uint64_t kNoKey = ~0ull;
constexpr int kMaxCluster = 16;
constexpr int kMaxGridClusters = 1024;  // clusters of one single-instance launch
constexpr int kMaxThreads = 512;  // per CTA; leaves 128 registers per thread
constexpr int kIdShift = 13;
constexpr uint32_t kIdMask = (1u << kIdShift) - 1u;
constexpr int kMaxMissions = 4095;
constexpr int kMaxNodes = 8192;
constexpr int kMaxVehicles = 1024;
constexpr int64_t kDefaultTimeoutNs = 1000000000ll;

// ------------------------------------------------------------------ layout ---------

// Per-node records. A node word packs the next node and the node's
// vehicle word: nv = next | vw << 13, vw = vehicle | plane << 10 | heli-only << 11.
//   R2[t] = {nv, removal delta}                       relocation, mission side
//   Y4[t] = {A row of prev(t), B row of t, leg prev(t) -> t, nv}   relocation, gap side
//   S4[t] = {nv, A row of prev(t), B row of next(t), slot cost}    swap side
//   D4[t] = {dep(prev t), arrive-by slack at t, slack at next(t), removal link ok}
//   PRV[t] previous node; FB[v] flight of vehicle v minus the duty cap;
//   RP[t]  (after FB) a relocation's delta on t's own route when t moves to another
//          route: removal delta plus lambda times the change of that route's overflow
//          (penalty mode), or whether the route stays within the cap (hard mode). Kept by
//          the batch and serving kernels, where it saves work in every relocation, and not
//          by the single-instance kernel, whose iterations wait on the record rewrite.
constexpr int kBufWordsPerNode = 15;

// Two table layouts. Small instances keep location x mission gather tables (int32):
//   A[t][l][m] = T_t[l][p_m] + T_t[p_m][d_m],  B[t][l][m] = T_t[d_m][l],
// row stride Mp words, so 32 lanes reading 32 consecutive missions hit 32 banks.
// Large instances ("big") keep the travel matrix itself in int16 (exact while every
// entry is below 2^15) with a row stride of Ls halves, Ls / 2 odd, so that random rows
// and random columns both spread over the banks; tabu stamps are int16 there too.
struct Layout {  // offsets in int32 words from the start of dynamic shared memory
  int A, B, tabu, cmat, wm, eloc, sloc, vtype, tyl, tym, st0, best, order, cnt, gend, gdep, gfl,
      glast, misc, mbar, warpkey, slots, gkey, total;
  int Mp, Np, Vp, buf, Ls;
  bool big;
};

__host__ __device__ inline int round_up(int x, int k) { return (x + k - 1) / k * k; }

__host__ __device__ inline Layout make_layout(int M, int V, int L, int nt, bool big, bool rp) {
  Layout y;
  y.big = big;
  y.Mp = round_up(M > 0 ? M : 1, 32);
  y.Np = round_up(M + V, 4);
  y.Vp = round_up(V, 4);
  y.buf = kBufWordsPerNode * y.Np + y.Vp + (rp ? y.Np : 0);  // R2 Y4 S4 D4 PRV, FB, RP
  y.Ls = round_up(L, 2);
  if ((y.Ls / 2) % 2 == 0) y.Ls += 2;
  int o = 0;
  if (big) {
    y.A = o;     o += round_up(nt * L * y.Ls / 2, 4);  // int16 travel matrix
    y.B = y.A;
    y.tabu = o;  o += round_up(V * y.Mp / 2, 4);      // int16 stamps
  } else {
    y.A = o;     o += nt * L * y.Mp;
    y.B = o;     o += nt * L * y.Mp;
    y.tabu = o;  o += V * y.Mp;
  }
  y.cmat = o;    o += nt * y.Mp;
  y.wm = o;      o += y.Mp;
  y.eloc = o;    o += round_up(M + V + 3, 4);  // + 3: quads of missions read up to M + 2
  y.sloc = o;    o += round_up(M + V + 3, 4);
  y.vtype = o;   o += y.Vp;
  y.tyl = o;     o += y.Vp;
  y.tym = o;     o += y.Vp;
  y.st0 = o;     o += y.buf;
  y.best = o;    o += y.Np;
  y.order = o;   o += y.Mp;
  y.cnt = o;     o += y.Mp;
  y.gend = o;    o += y.Vp;
  y.gdep = o;    o += y.Vp;
  y.gfl = o;     o += y.Vp;
  y.glast = o;   o += y.Vp;
  y.misc = o;    o += 16;
  y.mbar = o;    o += 2;  // one mbarrier (8 bytes; o is even here)
  o = round_up(o, 4);
  y.warpkey = o; o += 2 * 32;
  y.slots = o;   o += 2 * 2 * kMaxCluster;
  y.gkey = o;    o += 2 * 2;  // the grid's key, per slot buffer (several clusters)
  y.total = o;
  return y;
}

// ------------------------------------------------------------------ parameters -----

struct KParams {
  const int32_t* travel;
  const int32_t* veh_base;
  const int32_t* veh_type;
  const int32_t* pickup;
  const int32_t* delivery;
  const int32_t* heli_only;
  const int32_t* deadline;
  int32_t L, nt, V, M, cap, horizon;
  int32_t tenure, iterations, lambda, cluster;
  int32_t grid_clusters;  // clusters cooperating on the instance (1: one cluster)
  int32_t gslot_stride;   // words (uint64) between the two global slot buffers
  uint64_t* gslots;       // [2][gslot_stride] keys of the clusters (grid_clusters > 1), zeroed
  int32_t test_withhold;  // the last CTA (cluster) does not publish its first key (tests the timeout)
  int64_t timeout_ns;
  Layout lay;
  const int32_t* init_off;
  const int32_t* init_route;
  const int32_t* tabu_in;
  int32_t dbg_it, dbg_zbest;
  int32_t* out_off;
  int32_t* out_route;
  int32_t* out_flight;
  int32_t* out_over;
  int32_t* info;
  uint32_t* traj_move;
  int32_t* traj_z;
  int32_t* dbg_delta;
  uint8_t* dbg_flags;
  uint32_t* dbg_id;
  unsigned long long* dbg_key;
};

// ------------------------------------------------------------------ PTX helpers ----

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// CTAs in this CTA's cluster as launched (1 without a cluster launch).
__device__ __forceinline__ uint32_t cluster_ctas() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

// The launch has the shape the parameters describe: C CTAs per cluster and `ctas` CTAs
// in all, in a one-dimensional grid. Kernels check this before any access to a peer's
// shared memory, whose address would not exist in a launch of another shape (for
// instance one replayed without its cluster attribute).
__device__ __forceinline__ bool launch_shape_ok(int C, int ctas) {
  return static_cast<int>(cluster_ctas()) == C && (ctas <= 0 || static_cast<int>(gridDim.x) == ctas) &&
         gridDim.y == 1 && gridDim.z == 1;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

// The same cluster barrier without .aligned: for code where the threads of a warp may
// arrive from different paths (the warp is also synchronised first).
__device__ __forceinline__ void cluster_sync_unaligned() {
  __syncwarp();
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ uint32_t mapa_rank(uint32_t local_addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_addr), "r"(rank));
  return r;
}

// Store into a peer CTA's shared memory (relaxed, cluster scope).
__device__ __forceinline__ void st_peer_u64(uint32_t cluster_addr, uint64_t v) {
  asm volatile("st.relaxed.cluster.shared::cluster.u64 [%0], %1;" ::"r"(cluster_addr), "l"(v) : "memory");
}

// Load a 32-bit word from a peer CTA's shared memory (ordered by a cluster barrier).
__device__ __forceinline__ int ld_peer_i32(uint32_t cluster_addr) {
  int v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(cluster_addr) : "memory");
  return v;
}

// Store into this CTA's shared memory for its other warps (relaxed, CTA scope).
__device__ __forceinline__ void st_own_u64(uint32_t cta_addr, uint64_t v) {
  asm volatile("st.relaxed.cta.shared::cta.u64 [%0], %1;" ::"r"(cta_addr), "l"(v) : "memory");
}

// Load from this CTA's shared memory, observing peers' relaxed stores.
__device__ __forceinline__ uint64_t ld_own_u64(uint32_t cta_addr) {
  uint64_t v;
  asm volatile("ld.relaxed.cluster.shared::cta.u64 %0, [%1];" : "=l"(v) : "r"(cta_addr) : "memory");
  return v;
}

// ---- bulk copies global -> shared completing on an mbarrier (compact layout staging)
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// before the barrier's memory serves anything else (the next instance of a persistent
// launch may lay shared memory out differently)
__device__ __forceinline__ void mbar_inval(uint32_t bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bytes from global src into this CTA's shared dst (both 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// OR of a flag into a word of another CTA's shared memory
__device__ __forceinline__ void red_or_peer(uint32_t cluster_addr, uint32_t v) {
  asm volatile("red.shared::cluster.or.b32 [%0], %1;" ::"r"(cluster_addr), "r"(v) : "memory");
}

// Keys between the clusters of one instance go through global memory (L2): relaxed
// stores and loads at GPU scope, each a single 64-bit word that carries its own tag.
__device__ __forceinline__ void st_relaxed_gpu_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_gpu_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Instance inputs are read through L2 only (ld.global.cg): a persistent launch reuses
// request slots whose new contents arrive by copy while it runs, and L1 is not kept
// coherent with those writes. These reads happen outside the iteration loop.
__device__ __forceinline__ int gin(const int32_t* p) { return __ldcg(p); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ------------------------------------------------------------------ keys -----------

// Bits 26-29 of every move id are zero (R ids < 2^26; S ids use bit 31 and bits
// 0-25), so keys crossing the cluster carry an iteration tag there: 8 | ((it >> 1) & 7).
// Slots start at 0 (tag 0), and consecutive uses of a slot buffer carry different tags.
constexpr uint64_t kTagMask = 0xFull << 26;
// Bit 30 is zero in every move id too. In a key broadcast to the CTAs of a cluster it
// means "the exchange between clusters gave up" (with a high word of all ones).
constexpr uint64_t kFailBit = 1ull << 30;
__device__ __forceinline__ uint64_t iter_tag(int it) {
  return static_cast<uint64_t>(8 | ((it >> 1) & 7)) << 26;
}

__device__ __forceinline__ uint64_t pack_key(int32_t d, uint32_t id) {
  return (static_cast<uint64_t>(static_cast<uint32_t>(d) ^ 0x80000000u) << 32) | id;
}
__device__ __forceinline__ int32_t key_delta(uint64_t k) {
  return static_cast<int32_t>(static_cast<uint32_t>(k >> 32) ^ 0x80000000u);
}

__device__ __forceinline__ uint64_t warp_min_key(uint64_t k) {
  const uint32_t hi = static_cast<uint32_t>(k >> 32), lo = static_cast<uint32_t>(k);
  const uint32_t mhi = __reduce_min_sync(0xffffffffu, hi);
  const uint32_t mlo = __reduce_min_sync(0xffffffffu, hi == mhi ? lo : 0xffffffffu);
  return (static_cast<uint64_t>(mhi) << 32) | mlo;
}

__device__ __forceinline__ uint64_t min_u64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int32_t pos0(int32_t x) { return x > 0 ? x : 0; }

// ------------------------------------------------------------------ shared state ---

// All state lives in dynamic shared memory and is addressed as word offsets into this
// one array, so every access compiles to a shared-memory load or store.
extern __shared__ __align__(16) int32_t g_smem[];

struct Arr {  // an int32 array in shared memory
  int off;
  __device__ __forceinline__ int32_t& operator[](int i) const { return g_smem[off + i]; }
};

struct State {  // the per-node records (see the layout notes)
  int base, np, vp;
  __device__ __forceinline__ int2* r2() const { return reinterpret_cast<int2*>(g_smem + base); }
  __device__ __forceinline__ int4* y4() const { return reinterpret_cast<int4*>(g_smem + base + 2 * np); }
  __device__ __forceinline__ int4* s4() const { return reinterpret_cast<int4*>(g_smem + base + 6 * np); }
  __device__ __forceinline__ int4* d4() const { return reinterpret_cast<int4*>(g_smem + base + 10 * np); }
  __device__ __forceinline__ int32_t* prv() const { return g_smem + base + 14 * np; }
  __device__ __forceinline__ int32_t* fb() const { return g_smem + base + 15 * np; }
  __device__ __forceinline__ int32_t* rp() const { return g_smem + base + 15 * np + vp; }
  __device__ __forceinline__ int32_t& nv(int t) const { return g_smem[base + 2 * t]; }
};

struct Smem {
  Arr A, B, tabu, cmat, wm, eloc, sloc, vtype, tyl, tym, best, order, cnt, gend, gdep, gfl, glast, misc;
  int st0, buf, np, vp;
  int warpkey_off, slots_off, gkey_off;
  __device__ __forceinline__ State records() const { return State{st0, np, vp}; }  // the per-node records
  __device__ __forceinline__ uint64_t* warpkey() const {
    return reinterpret_cast<uint64_t*>(g_smem + warpkey_off);
  }
  __device__ __forceinline__ uint64_t* slots() const { return reinterpret_cast<uint64_t*>(g_smem + slots_off); }
  __device__ __forceinline__ uint64_t* gkey() const { return reinterpret_cast<uint64_t*>(g_smem + gkey_off); }
};

__device__ inline Smem carve(const Layout& y) {
  Smem s;
  s.A = Arr{y.A};
  s.B = Arr{y.B};
  s.tabu = Arr{y.tabu};
  s.cmat = Arr{y.cmat};
  s.wm = Arr{y.wm};
  s.eloc = Arr{y.eloc};
  s.sloc = Arr{y.sloc};
  s.vtype = Arr{y.vtype};
  s.tyl = Arr{y.tyl};
  s.tym = Arr{y.tym};
  s.st0 = y.st0;
  s.buf = y.buf;
  s.np = y.Np;
  s.vp = y.Vp;
  s.best = Arr{y.best};
  s.order = Arr{y.order};
  s.cnt = Arr{y.cnt};
  s.gend = Arr{y.gend};
  s.gdep = Arr{y.gdep};
  s.gfl = Arr{y.gfl};
  s.glast = Arr{y.glast};
  s.misc = Arr{y.misc};
  s.warpkey_off = y.warpkey;
  s.slots_off = y.slots;
  s.gkey_off = y.gkey;
  return s;
}

// misc slots
enum { MISC_BAD = 0, MISC_MAXT, MISC_Z0, MISC_GREEDY_FAIL, MISC_CSR_BAD, MISC_STAGE_FAIL };

struct Ctx {  // per-launch constants every thread keeps in registers
  int M, V, N, L, Mp, cap, horizon, lam;
  int heli;  // some mission is heli-only
};

// Table access for either layout. A row handle is (type offset + location) times the
// row unit: Mp words for the gather tables, 1 (a row index) for the int16 matrix.
template <bool BIG>
struct Tab {
  int A, B, tabu_off, cmat, eloc, sloc;
  int Mp, L, Ls;
  __device__ __forceinline__ int row(int tyl, int loc) const { return BIG ? tyl + loc : (tyl + loc) * Mp; }
  __device__ __forceinline__ int t16(int i) const { return reinterpret_cast<const int16_t*>(g_smem + A)[i]; }
  // A[row][m]: fly from the row's location to m's pickup, then m's own leg.
  __device__ __forceinline__ int a(int r, int m) const {
    if (BIG) return t16(r * Ls + g_smem[sloc + m]) + g_smem[cmat + (r >= L ? Mp : 0) + m];
    return g_smem[A + r + m];
  }
  // B[row][m]: from m's delivery to the row's location.
  __device__ __forceinline__ int b(int r, int m) const {
    if (BIG) {
      const int tyl = r >= L ? L : 0;
      return t16((tyl + g_smem[eloc + m]) * Ls + (r - tyl));
    }
    return g_smem[B + r + m];
  }
  // Entries of missions m0 and m0 + 1 (m0 even). The per-mission arrays start on 16-byte
  // boundaries (every layout offset is a multiple of 4 words), so the pair's locations
  // and legs come in single 64-bit loads.
  __device__ __forceinline__ int2 a2(int r, int m0) const {
    if (BIG) {
      const int2 s = *reinterpret_cast<const int2*>(g_smem + sloc + m0);
      const int2 cm = *reinterpret_cast<const int2*>(g_smem + cmat + (r >= L ? Mp : 0) + m0);
      const int base = r * Ls;
      return make_int2(t16(base + s.x) + cm.x, t16(base + s.y) + cm.y);
    }
    return *reinterpret_cast<const int2*>(g_smem + A + r + m0);
  }
  __device__ __forceinline__ int2 b2(int r, int m0) const {
    if (BIG) {
      const int tyl = r >= L ? L : 0;
      const int2 e = *reinterpret_cast<const int2*>(g_smem + eloc + m0);
      const int col = r - tyl;
      return make_int2(t16((tyl + e.x) * Ls + col), t16((tyl + e.y) * Ls + col));
    }
    return *reinterpret_cast<const int2*>(g_smem + B + r + m0);
  }
  // Entries of missions m0 .. m0 + 3 (m0 a multiple of 4), by 128-bit loads.
  __device__ __forceinline__ int4 a4(int r, int m0) const {
    if (BIG) {
      const int4 s = *reinterpret_cast<const int4*>(g_smem + sloc + m0);
      const int4 cm = *reinterpret_cast<const int4*>(g_smem + cmat + (r >= L ? Mp : 0) + m0);
      const int base = r * Ls;
      return make_int4(t16(base + s.x) + cm.x, t16(base + s.y) + cm.y, t16(base + s.z) + cm.z,
                       t16(base + s.w) + cm.w);
    }
    return *reinterpret_cast<const int4*>(g_smem + A + r + m0);
  }
  __device__ __forceinline__ int4 b4(int r, int m0) const {
    if (BIG) {
      const int tyl = r >= L ? L : 0;
      const int4 e = *reinterpret_cast<const int4*>(g_smem + eloc + m0);
      const int col = r - tyl;
      return make_int4(t16((tyl + e.x) * Ls + col), t16((tyl + e.y) * Ls + col), t16((tyl + e.z) * Ls + col),
                       t16((tyl + e.w) * Ls + col));
    }
    return *reinterpret_cast<const int4*>(g_smem + B + r + m0);
  }
  __device__ __forceinline__ int4 tabu4(int v, int m0) const {
    if (BIG) {
      const short4 w = *reinterpret_cast<const short4*>(reinterpret_cast<const int16_t*>(g_smem + tabu_off) +
                                                         v * Mp + m0);
      return make_int4(w.x, w.y, w.z, w.w);
    }
    return *reinterpret_cast<const int4*>(g_smem + tabu_off + v * Mp + m0);
  }
  __device__ __forceinline__ int tabu(int v, int m) const {
    if (BIG) return reinterpret_cast<const int16_t*>(g_smem + tabu_off)[v * Mp + m];
    return g_smem[tabu_off + v * Mp + m];
  }
  __device__ __forceinline__ int2 tabu2(int v, int m0) const {  // m0 even
    if (BIG) {
      const short2 w = *reinterpret_cast<const short2*>(reinterpret_cast<const int16_t*>(g_smem + tabu_off) +
                                                         v * Mp + m0);
      return make_int2(w.x, w.y);
    }
    return *reinterpret_cast<const int2*>(g_smem + tabu_off + v * Mp + m0);
  }
  __device__ __forceinline__ void set_tabu(int v, int m, int x) const {
    if (BIG) reinterpret_cast<int16_t*>(g_smem + tabu_off)[v * Mp + m] = static_cast<int16_t>(x);
    else g_smem[tabu_off + v * Mp + m] = x;
  }
};

template <bool BIG>
__device__ __forceinline__ Tab<BIG> make_tab(const Layout& y, int L) {
  Tab<BIG> t;
  t.A = y.A;
  t.B = y.B;
  t.tabu_off = y.tabu;
  t.cmat = y.cmat;
  t.eloc = y.eloc;
  t.sloc = y.sloc;
  t.Mp = y.Mp;
  t.L = L;
  t.Ls = y.Ls;
  return t;
}

constexpr int kNodeMask = 0x1FFF;  // next-node field of a node word
__device__ __forceinline__ int nv_next(int nv) { return nv & kNodeMask; }
__device__ __forceinline__ int nv_vw(int nv) { return (nv >> 13) & 0xFFF; }
__device__ __forceinline__ int nv_veh(int nv) { return (nv >> 13) & 0x3FF; }
__device__ __forceinline__ int vw_veh(int vw) { return vw & 0x3FF; }
__device__ __forceinline__ int vw_plane(int vw) { return (vw >> 10) & 1; }
// the vehicle part of `from` with the heli-only bit of `own`
__device__ __forceinline__ int vw_move(int from, int own) { return (from & 0x7FF) | (own & 0x800); }

// Write every record of node t into S from its links (nx, pv), its vehicle
// word vw and the flight f2 of that vehicle.
template <bool PEN, bool DL, bool BIG, bool RP>
__device__ __forceinline__ void write_records(const Smem& sm, const Tab<BIG>& tb, const State& S, const Ctx& c,
                                              int t, int nx, int pv, int vw, int f2) {
  // Every load comes before the first store: the stores go to the same shared array, so
  // the compiler could not move a load above one of them.
  const int plane = vw_plane(vw);
  const int tyl = plane * c.L, tym = plane * c.Mp;
  const int rowA = tb.row(tyl, sm.eloc[pv]);
  const int rowB = tb.row(tyl, sm.sloc[t]);
  const int nv = nx | (vw << 13);
  const int dep = (DL && pv < c.M) ? sm.wm[pv] : 0;
  if (t < c.M) {
    const int rowBn = tb.row(tyl, sm.sloc[nx]);
    const int aT = tb.a(rowA, t);
    const int bT = tb.b(rowBn, t);
    const int slot = aT + bT;
    const int ct = sm.cmat[tym + t];
    const int cn = nx < c.M ? sm.cmat[tym + nx] : 0;
    const int leg = nx < c.M ? tb.a(rowA, nx) - cn : (pv < c.M ? tb.b(rowBn, pv) : 0);
    const int wt = DL ? sm.wm[t] : 0;
    const int wn = DL ? (nx < c.M ? sm.wm[nx] : c.horizon) : 0;
    const int rem = leg - slot;
    S.prv()[t] = pv;
    S.r2()[t] = make_int2(nv, rem);
    if (RP) {
      const int fm = f2 - c.cap;
      S.rp()[t] = PEN ? rem + c.lam * (pos0(fm + rem) - pos0(fm)) : (fm + rem <= 0 ? 1 : 0);
    }
    S.y4()[t] = make_int4(rowA, rowB, aT - ct, nv);
    S.s4()[t] = make_int4(nv, rowA, rowBn, slot);
    if (DL) S.d4()[t] = make_int4(dep, wt - ct, wn - cn, (dep + leg + cn <= wn) ? 1 : 0);
  } else {
    const int inleg = (pv == t) ? 0 : tb.b(rowB, pv);
    S.prv()[t] = pv;
    S.r2()[t] = make_int2(nv, 0);
    S.y4()[t] = make_int4(rowA, rowB, inleg, nv);
    S.s4()[t] = make_int4(nv, 0, 0, 0);
    S.fb()[t - c.M] = f2 - c.cap;
    if (DL) S.d4()[t] = make_int4(dep, c.horizon, 0, 1);
  }
}

__device__ __forceinline__ uint8_t move_flags(bool feas, bool tabu, bool asp, bool adm) {
  return static_cast<uint8_t>((feas ? 1 : 0) | (tabu ? 2 : 0) | (asp ? 4 : 0) | (adm ? 8 : 0));
}

// Relocation R(m, y): take m out, put it immediately before node y. The inputs are
// already loaded: m's node word, removal delta and RP record, the gap record g of y, the
// table entries a = A[row of prev(y)][m], b = B[row of y][m], y's vehicle slack fy and
// the tabu stamp of (m, vehicle of y). zrel = z_best - Z, so the move aspires when
// delta < zrel (Z + delta < z_best). An admissible move's key replaces acc when smaller.
// HELI: the instance has heli-only missions (else the compatibility test is always true).
template <bool PEN, bool DL, bool DEBUG, bool RP, bool HELI>
__device__ __forceinline__ void reloc_one(const Smem& sm, const State& S, const Ctx& c, int y, int m, int nvm,
                                          int rem, int rp, const int4& g, int a, int b, int fy, int stamp, int it,
                                          int zrel, const KParams& P, uint64_t& acc) {
  const bool valid = (y != m) && (y != nv_next(nvm));
  const int vm = nv_veh(nvm), vy = nv_veh(g.w);
  const int ins = a + b - g.z;
  const int d = rem + ins;
  // Same route: one flight changes by d. Different routes: the source's flight by rem
  // (its part of the delta is m's RP record where kept), the target's by ins. Both are
  // computed and selected, so lanes never diverge.
  const bool same = vm == vy;
  int delta;
  bool feas;
  if (RP) {
    const int grow = same ? d : ins;  // change of the target route's flight
    if (PEN) {
      delta = (same ? d : rp + ins) + c.lam * (pos0(fy + grow) - pos0(fy));
      feas = true;
    } else {
      delta = d;
      feas = (fy + grow <= 0) && (same || rp != 0);
    }
  } else {
    const int fm = S.fb()[vm];
    if (PEN) {
      const int pen = same ? pos0(fy + d) : pos0(fm + rem) - pos0(fm) + pos0(fy + ins);
      delta = d + c.lam * (pen - pos0(fy));
      feas = true;
    } else {
      delta = d;
      feas = same ? (fy + d <= 0) : ((fm + rem <= 0) && (fy + ins <= 0));
    }
  }
  if (HELI) feas = feas && !((nvm >> 24) & (g.w >> 23) & 1);  // heli-only m onto a plane
  if (DL) {
    const int4 dy = S.d4()[y];
    const int w = sm.wm[m];
    feas = feas && (dy.x + a <= w) && (w + b <= dy.y) && S.d4()[m].w;
  }
  const bool tabu = stamp >= it;
  const bool asp = delta < zrel;
  const bool adm = valid && feas && (!tabu || asp);
  const uint32_t id = (static_cast<uint32_t>(m) << kIdShift) | static_cast<uint32_t>(y);
  if (DEBUG && valid) {
    const int64_t idx = static_cast<int64_t>(m) * (c.N - 2) + y - (y > m) - (y > nv_next(nvm));
    P.dbg_delta[idx] = delta;
    P.dbg_flags[idx] = move_flags(feas, tabu, asp, adm);
    if (P.dbg_id) P.dbg_id[idx] = id;
  }
  const uint64_t k = pack_key(delta, id);
  if (adm && k < acc) acc = k;
}

// Relocations of the mission pair (m0, m0 + 1), m0 even, before node y: every load
// serves both (64-bit loads of consecutive table and record entries).
template <bool PEN, bool DL, bool DEBUG, bool BIG, bool RP, bool HELI>
__device__ __forceinline__ void eval_relocate_pair(const Smem& sm, const Tab<BIG>& tb, const State& S, const Ctx& c,
                                                   int y, int m0, int it, int zrel, const KParams& P, uint64_t& acc) {
  const int4 rr = *reinterpret_cast<const int4*>(S.r2() + m0);  // {nv, rem} of m0 and m0 + 1
  const int2 rp = RP ? *reinterpret_cast<const int2*>(S.rp() + m0) : make_int2(0, 0);
  const int4 g = S.y4()[y];  // A row, B row, leg into y, node word of y
  const int vy = nv_veh(g.w);
  const int2 a2 = tb.a2(g.x, m0);
  const int2 b2 = tb.b2(g.y, m0);
  const int2 st = tb.tabu2(vy, m0);
  const int fy = S.fb()[vy];
  reloc_one<PEN, DL, DEBUG, RP, HELI>(sm, S, c, y, m0, rr.x, rr.y, rp.x, g, a2.x, b2.x, fy, st.x, it, zrel, P, acc);
  if (m0 + 1 < c.M)
    reloc_one<PEN, DL, DEBUG, RP, HELI>(sm, S, c, y, m0 + 1, rr.z, rr.w, rp.y, g, a2.y, b2.y, fy, st.y, it, zrel, P,
                                        acc);
}

// Relocations of missions m0 .. m0 + 3 (m0 a multiple of 4) before node y, for the batch
// and serving kernels: y's gap record, vehicle, flight and tabu row serve four moves, and
// the table rows, records and stamps of the four missions come in 128-bit loads.
template <bool PEN, bool DL, bool BIG, bool HELI>
__device__ __forceinline__ void eval_relocate_quad(const Smem& sm, const Tab<BIG>& tb, const State& S, const Ctx& c,
                                                   int y, int m0, int it, int zrel, const KParams& P, uint64_t& acc) {
  const int4 r01 = *reinterpret_cast<const int4*>(S.r2() + m0);      // {nv, rem} of m0, m0 + 1
  const int4 r23 = *reinterpret_cast<const int4*>(S.r2() + m0 + 2);  // and of m0 + 2, m0 + 3
  const int4 rp = *reinterpret_cast<const int4*>(S.rp() + m0);
  const int4 g = S.y4()[y];  // A row, B row, leg into y, node word of y
  const int vy = nv_veh(g.w);
  const int4 a4 = tb.a4(g.x, m0);
  const int4 b4 = tb.b4(g.y, m0);
  const int4 st = tb.tabu4(vy, m0);
  const int fy = S.fb()[vy];
  reloc_one<PEN, DL, false, true, HELI>(sm, S, c, y, m0, r01.x, r01.y, rp.x, g, a4.x, b4.x, fy, st.x, it, zrel, P, acc);
  if (m0 + 1 < c.M)
    reloc_one<PEN, DL, false, true, HELI>(sm, S, c, y, m0 + 1, r01.z, r01.w, rp.y, g, a4.y, b4.y, fy, st.y, it, zrel,
                                          P, acc);
  if (m0 + 2 < c.M)
    reloc_one<PEN, DL, false, true, HELI>(sm, S, c, y, m0 + 2, r23.x, r23.y, rp.z, g, a4.z, b4.z, fy, st.z, it, zrel,
                                          P, acc);
  if (m0 + 3 < c.M)
    reloc_one<PEN, DL, false, true, HELI>(sm, S, c, y, m0 + 3, r23.z, r23.w, rp.w, g, a4.w, b4.w, fy, st.w, it, zrel,
                                          P, acc);
}

// Cost parts of swap S(a, b), each mission taking the other's place: t1 = fly from the
// end of a's predecessor to b's pickup plus b's own leg, t2 = from b's delivery to a's
// successor's start, t3 and t4 the same for a in b's place. When a and b are neighbours
// the predecessor or successor is the other mission itself (its delivery row is used).
struct SwapParts {
  int4 sa, sb;
  int t1, t2, t3, t4;
  bool adjA, adjB;
};

template <bool BIG>
__device__ __forceinline__ SwapParts swap_parts(const Smem& sm, const Tab<BIG>& tb, const State& S, const Ctx& c,
                                                int a, int b) {
  SwapParts q;
  q.sa = S.s4()[a];
  q.sb = S.s4()[b];
  q.adjA = nv_next(q.sa.x) == b;  // a immediately before b
  q.adjB = nv_next(q.sb.x) == a;  // b immediately before a
  // A row of a mission's own delivery (needed only next to the other mission)
  const int rowEa = q.adjB ? tb.row(vw_plane(nv_vw(q.sa.x)) * c.L, sm.eloc[a]) : 0;
  const int rowEb = q.adjA ? tb.row(vw_plane(nv_vw(q.sb.x)) * c.L, sm.eloc[b]) : 0;
  q.t1 = tb.a(q.adjB ? rowEa : q.sa.y, b);
  q.t2 = tb.b(q.sa.z, q.adjA ? a : b);
  q.t3 = tb.a(q.adjA ? rowEb : q.sb.y, a);
  q.t4 = tb.b(q.sb.z, q.adjB ? b : a);
  return q;
}

// Swap S(a, b): the two missions exchange places. Aspiration and the key as in reloc_one.
// FAR: the main pass over every pair of the batch and serving kernels, which takes the
// cost parts of two missions that are not neighbours (no delivery rows, no selects) and
// leaves neighbouring pairs out; those are the pairs (t, next t) of their neighbour pass.
// FAR = false handles any pair whole (the single-instance kernel's pass over every pair,
// and the neighbour pass).
template <bool PEN, bool DL, bool DEBUG, bool BIG, bool HELI, bool FAR>
__device__ __forceinline__ void eval_swap(const Smem& sm, const Tab<BIG>& tb, const State& S, const Ctx& c, int a,
                                          int b, int it, int zrel, const KParams& P, uint64_t& acc) {
  SwapParts q;
  bool near = false;
  if (FAR) {
    q.sa = S.s4()[a];
    q.sb = S.s4()[b];
    near = nv_next(q.sa.x) == b || nv_next(q.sb.x) == a;
    q.adjA = q.adjB = false;
    q.t1 = tb.a(q.sa.y, b);
    q.t2 = tb.b(q.sa.z, b);
    q.t3 = tb.a(q.sb.y, a);
    q.t4 = tb.b(q.sb.z, a);
  } else {
    q = swap_parts<BIG>(sm, tb, S, c, a, b);
  }
  const int nva = q.sa.x, nvb = q.sb.x;
  const int va = nv_veh(nva), vb = nv_veh(nvb);
  const int da = q.t1 + q.t2 - q.sa.w;
  const int db = q.t3 + q.t4 - q.sb.w;
  const int fa = S.fb()[va], fb = S.fb()[vb];
  const bool same = va == vb;
  const int d = da + db;
  int delta;
  bool feas;
  if (PEN) {
    const int pen = same ? pos0(fa + d) - pos0(fa) : pos0(fa + da) - pos0(fa) + pos0(fb + db) - pos0(fb);
    delta = d + c.lam * pen;
    feas = true;
  } else {
    delta = d;
    feas = same ? (fa + d <= 0) : ((fa + da <= 0) && (fb + db <= 0));
  }
  if (HELI) feas = feas && !((((nva >> 24) & (nvb >> 23)) | ((nvb >> 24) & (nva >> 23))) & 1);
  if (DL) {
    const int4 xa = S.d4()[a], xb = S.d4()[b];
    const int wa = sm.wm[a], wb = sm.wm[b];
    const bool l1 = (q.adjB ? wa : xa.x) + q.t1 <= wb;
    const bool l2 = q.adjA || (wb + q.t2 <= xa.z);
    const bool l3 = (q.adjA ? wb : xb.x) + q.t3 <= wa;
    const bool l4 = q.adjB || (wa + q.t4 <= xb.z);
    feas = feas && l1 && l2 && l3 && l4;
  }
  const bool tabu = (tb.tabu(vb, a) >= it) || (tb.tabu(va, b) >= it);
  const bool asp = delta < zrel;
  const bool adm = !near && feas && (!tabu || asp);
  const int m1 = a < b ? a : b, m2 = a < b ? b : a;
  const uint32_t id = kSwapBit | (static_cast<uint32_t>(m1) << kIdShift) | static_cast<uint32_t>(m2);
  if (DEBUG && !near) {
    const int64_t rtot = static_cast<int64_t>(c.M) * (c.N - 2);
    const int64_t idx = rtot + static_cast<int64_t>(m1) * (2 * c.M - m1 - 1) / 2 + (m2 - m1 - 1);
    P.dbg_delta[idx] = delta;
    P.dbg_flags[idx] = move_flags(feas, tabu, asp, adm);
    if (P.dbg_id) P.dbg_id[idx] = id;
  }
  const uint64_t k = pack_key(delta, id);
  if (adm && k < acc) acc = k;
}

// One thread's share of the evaluation (see the main loop for the item list and how its
// coordinates advance); returns the least admissible key among its moves.
struct ItemCursor {
  int r_y, r_h, s_j, s_row, s_a;  // first relocation item (y, h) and swap item (j, row, a)
  int Gq, Gr, Sq, Sr, G, H, Sn;   // grid stride in both coordinate systems, list sizes
  int n_k;                        // first item of the neighbour pass (mission t)
};

template <bool PEN, bool DL, bool DEBUG, bool BIG, bool RP, bool HELI>
__device__ __forceinline__ uint64_t eval_items(const Smem& sm, const Tab<BIG>& tb, const State& S, const Ctx& c,
                                               const ItemCursor& q, int it, int zrel, const KParams& P) {
  uint64_t key = kNoKey;
  for (int y = q.r_y, h = q.r_h; y < c.N;) {
    if (RP) eval_relocate_quad<PEN, DL, BIG, HELI>(sm, tb, S, c, y, 4 * h, it, zrel, P, key);
    else eval_relocate_pair<PEN, DL, DEBUG, BIG, RP, HELI>(sm, tb, S, c, y, 2 * h, it, zrel, P, key);
    h += q.Gr;
    y += q.Gq;
    if (h >= q.H) {
      h -= q.H;
      ++y;
    }
  }
  for (int j = q.s_j, row = q.s_row, a = q.s_a; j < q.Sn; j += q.G) {
    int b = a + row + 1;
    if (b >= c.M) b -= c.M;
    eval_swap<PEN, DL, DEBUG, BIG, HELI, RP>(sm, tb, S, c, a, b, it, zrel, P, key);
    a += q.Sr;
    row += q.Sq;
    if (a >= c.M) {
      a -= c.M;
      ++row;
    }
  }
  // Swaps of neighbours, t and its successor (the batch and serving kernels only, which
  // are bound by instruction issue: the main pass then takes the short form of every
  // pair; the single-instance kernel, bound by the latency of its slowest warp, keeps one
  // pass over the pairs with the neighbour case inside).
  if (RP) {
    for (int t = q.n_k; t < c.M; t += q.G) {
      const int u = nv_next(S.nv(t));
      if (u < c.M) eval_swap<PEN, DL, DEBUG, BIG, HELI, false>(sm, tb, S, c, t, u, it, zrel, P, key);
    }
  }
  return key;
}

// Flight after move `id` of the source route (src) or of the target route (!src): the
// route's flight from FB plus the move's change of it, from the same records and table
// entries the evaluators use. A move inside one route changes it by the whole delta.
template <bool BIG>
__device__ __forceinline__ int moved_flight(const Smem& sm, const Tab<BIG>& tb, const State& S, const Ctx& c,
                                            uint32_t id, bool src) {
  if (!(id & kSwapBit)) {
    const int m = static_cast<int>(id >> kIdShift), y = static_cast<int>(id & kIdMask);
    const int2 r = S.r2()[m];
    const int4 g = S.y4()[y];
    const int va = nv_veh(r.x), vb = nv_veh(g.w);
    const int ins = tb.a(g.x, m) + tb.b(g.y, m) - g.z;
    const int f = S.fb()[src ? va : vb] + c.cap;
    if (va == vb) return f + r.y + ins;
    return src ? f + r.y : f + ins;
  }
  const int a = static_cast<int>((id >> kIdShift) & kIdMask), b = static_cast<int>(id & kIdMask);
  const SwapParts q = swap_parts<BIG>(sm, tb, S, c, a, b);
  const int va = nv_veh(q.sa.x), vb = nv_veh(q.sb.x);
  const int da = q.t1 + q.t2 - q.sa.w;
  const int db = q.t3 + q.t4 - q.sb.w;
  const int f = S.fb()[src ? va : vb] + c.cap;
  if (va == vb) return f + da + db;
  return src ? f + da : f + db;
}

// ------------------------------------------------------------------ the kernel -----

// The compact layout's int16 matrix, row t*L + r of layer t at T16 + (t*L + r) * Ls, zero
// padded, built from the int32 input through a staging buffer: the record buffer, which
// nothing uses before the prologue writes the records. When the input is 16-byte aligned
// its words go by bulk copies completing on an mbarrier, in chunks the size of the
// buffer; every CTA copies every chunk into its own shared memory (the cluster reads the
// matrix from L2 C times; 230 KB per CTA once per solve). A block barrier after each
// chunk keeps the buffer free until every thread has converted it. Every wait is bounded
// by P.timeout_ns. With C > 1 CTAs the outcome is made the same in every CTA: a CTA whose
// copy gave up ORs a flag into rank 0's shared memory, and every CTA reads it after a
// cluster barrier. Entries are checked (>= 0) and their maximum taken on the way.
// Returns true on a timeout (in every CTA of the cluster when one timed out).
__device__ __forceinline__ bool stage_matrix16(const KParams& P, const Layout& lay, int C, int& bad, int& maxT) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int L = P.L, nt = P.nt, Ls = lay.Ls, pad = lay.Ls - P.L;
  int16_t* T16 = reinterpret_cast<int16_t*>(g_smem + lay.A);
  for (int i = tid; i < nt * L * pad; i += nthr) {
    const int r = i / pad;
    T16[r * Ls + L + (i - r * pad)] = 0;
  }
  auto put = [&](int g, int x) {
    bad |= x < 0;
    maxT = x > maxT ? x : maxT;
    const int r = g / L;
    T16[r * Ls + (g - r * L)] = static_cast<int16_t>(x);
  };
  const int words = nt * L * L;
  const bool aligned = (reinterpret_cast<uintptr_t>(P.travel) & 15u) == 0;
  const int bulk = aligned ? (words & ~3) : 0;  // words that go by bulk copies (16-byte units)
  for (int g = bulk + tid; g < words; g += nthr) put(g, gin(P.travel + g));
  const uint32_t fail_addr = smem_u32(&g_smem[lay.misc + MISC_STAGE_FAIL]);
  // Every CTA has zeroed its misc words (prologue 1) before any peer may OR into them.
  if (C > 1) cluster_sync_unaligned();
  bool gave_up = false;  // this CTA's wait ran out
  uint32_t phase = 0;
  if (bulk > 0) {
    int32_t* stage = g_smem + lay.st0;
    const int cap = lay.buf & ~3;
    const uint32_t bar = smem_u32(g_smem + lay.mbar);
    if (tid == 0) {
      mbar_init(bar, 1);
      mbar_fence_init();
    }
    __syncthreads();
    for (int c0 = 0; c0 < bulk; c0 += cap, phase ^= 1u) {
      const int n = bulk - c0 < cap ? bulk - c0 : cap;
      if (tid == 0) {
        // the block's reads of the previous chunk come before the copy overwrites it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar, static_cast<uint32_t>(n) * 4u);
        bulk_g2s(smem_u32(stage), P.travel + c0, static_cast<uint32_t>(n) * 4u, bar);
      }
      bool ok = mbar_try_wait(bar, phase);
      if (!ok) {
        const uint64_t t0 = global_ns();
        while (!(ok = mbar_try_wait(bar, phase))) {
          if (static_cast<int64_t>(global_ns() - t0) > P.timeout_ns) break;
        }
      }
      if (!__syncthreads_and(ok)) {
        gave_up = true;
        break;
      }
      for (int i = tid; i < n; i += nthr) put(c0 + i, stage[i]);
      __syncthreads();
    }
    if (gave_up) {  // let the copy still in flight land (bounded) before the buffer is reused
      const uint64_t t0 = global_ns();
      while (!mbar_try_wait(bar, phase) && static_cast<int64_t>(global_ns() - t0) < P.timeout_ns) {
      }
    }
    __syncthreads();  // nobody waits on the barrier after this
    if (tid == 0) mbar_inval(bar);
  }
  if (C == 1) return gave_up;
  if (gave_up && tid == 0) red_or_peer(mapa_rank(fail_addr, 0), 1u);
  cluster_sync_unaligned();
  const bool stop = ld_peer_i32(mapa_rank(fail_addr, 0)) != 0;
  cluster_sync_unaligned();  // nobody reads rank 0's flag after this
  return stop;
}

// One complete search (prologue, every iteration, epilogue) of the instance in P by
// the K clusters of C CTAs each (this CTA is `rank` in cluster `cid`), with shared
// memory laid out by lay. Every CTA holds the whole state and applies every move; CTA 0
// of cluster 0 writes the outputs.
template <bool PEN, bool DL, bool DEBUG, bool BIG, bool RP>
__device__ __forceinline__ void solve_one(const KParams& P, const Layout& lay, const int C, const int rank,
                                          const int K, const int cid) {
  const bool lead = rank == 0 && cid == 0;
  const Smem sm = carve(lay);
  const Tab<BIG> tb = make_tab<BIG>(lay, P.L);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  Ctx c;
  c.M = P.M;
  c.V = P.V;
  c.N = P.M + P.V;
  c.L = P.L;
  c.Mp = lay.Mp;
  c.cap = P.cap;
  c.horizon = P.horizon;
  c.lam = P.lambda;
  const int M = c.M, V = c.V, N = c.N, L = c.L, Mp = c.Mp, nt = P.nt;
  int status = ASCHED_OK;

  // ---- prologue 1: static per-mission / per-node data and validation
  if (tid < 16) sm.misc[tid] = 0;
  __syncthreads();
  int bad = 0, any_heli = 0;
  for (int i = tid; i < Mp; i += nthr) {
    if (i < M) {
      const int p = gin(P.pickup + i), d = gin(P.delivery + i);
      const int h = P.heli_only ? gin(P.heli_only + i) : 0;
      bad |= (p < 0) | (p >= L) | (d < 0) | (d >= L) | (p == d) | (h < 0) | (h > 1);
      any_heli |= h != 0;
      sm.wm[i] = P.deadline ? gin(P.deadline + i) : 0;
      sm.eloc[i] = d;
      sm.sloc[i] = p;
      sm.cnt[i] = 0;
    } else {
      sm.wm[i] = 0;
    }
  }
  for (int v = tid; v < V; v += nthr) {
    const int b = gin(P.veh_base + v);
    const int ty = P.veh_type ? gin(P.veh_type + v) : 0;
    bad |= (b < 0) | (b >= L) | (ty < 0) | (ty >= nt);
    sm.eloc[M + v] = b;
    sm.sloc[M + v] = b;
    sm.vtype[v] = ty;
    sm.tyl[v] = ty * L;
    sm.tym[v] = ty * Mp;
  }
  for (int i = N + tid; i < round_up(N + 3, 4); i += nthr) {  // padding read by quads of missions
    sm.eloc[i] = 0;
    sm.sloc[i] = 0;
  }
  int maxT = 0;
  if (!BIG) {  // the compact layout checks the matrix while it stages it (prologue 2)
    for (int i = tid; i < nt * L * L; i += nthr) {
      const int x = gin(P.travel + i);
      bad |= x < 0;
      maxT = x > maxT ? x : maxT;
    }
  }
  if (__syncthreads_or(bad)) status = ASCHED_E_INVALID;
  c.heli = __syncthreads_or(any_heli);
  if (BIG && status == ASCHED_OK) {
    // ---- prologue 1b: the int16 matrix, staged through shared memory by bulk copies,
    // checked as it is converted
    int tbad = 0;
    const bool timed_out = stage_matrix16(P, lay, C, tbad, maxT);
    if (__syncthreads_or(tbad)) status = ASCHED_E_INVALID;
    if (timed_out) status = ASCHED_E_TIMEOUT;  // the same in every CTA of the cluster
  }
  maxT = __reduce_max_sync(0xffffffffu, maxT);
  if (lane == 0) atomicMax(&sm.misc[MISC_MAXT], maxT);
  __syncthreads();
  if (BIG && status == ASCHED_OK && sm.misc[MISC_MAXT] > 32767) status = ASCHED_E_TOO_LARGE;
  if (status == ASCHED_OK) {
    // 2 (2M + V + 2) maxT (1 + lambda) < 2^31 keeps every int32 sum in range.
    const double bound = 2.0 * (2.0 * M + V + 2.0) * static_cast<double>(sm.misc[MISC_MAXT]) *
                         (1.0 + (PEN ? static_cast<double>(c.lam) : 0.0));
    if (!(bound < 2147483648.0)) status = ASCHED_E_OVERFLOW_GUARD;
  }

  // ---- prologue 2: gather tables, in-mission legs, tabu stamps, route ends
  const State S0 = sm.records();
  if (status == ASCHED_OK) {
    if (!BIG) {
      for (int i = tid; i < nt * L * Mp; i += nthr) {
        const int r = i / Mp, m = i - r * Mp;
        const int t = r / L, l = r - t * L;
        int av = 0, bv = 0;
        if (m < M) {
          const int32_t* T = P.travel + static_cast<int64_t>(t) * L * L;
          const int p = sm.sloc[m], d = sm.eloc[m];
          av = gin(T + l * L + p) + gin(T + p * L + d);
          bv = gin(T + d * L + l);
        }
        sm.A[i] = av;
        sm.B[i] = bv;
      }
    }
    for (int i = tid; i < nt * Mp; i += nthr) {
      const int t = i / Mp, m = i - t * Mp;
      int cv = 0;
      if (m < M) {
        const int32_t* T = P.travel + static_cast<int64_t>(t) * L * L;
        cv = gin(T + sm.sloc[m] * L + sm.eloc[m]);
      }
      sm.cmat[i] = cv;
    }
    for (int i = tid; i < V * Mp; i += nthr) {
      const int v = i / Mp, m = i - v * Mp;
      tb.set_tabu(v, m, (P.tabu_in && m < M) ? gin(P.tabu_in + static_cast<int64_t>(m) * V + v) : -1);
    }
    for (int v = tid; v < V; v += nthr) {
      S0.nv(M + v) = (M + v) | ((v | ((sm.vtype[v] != 0 ? 1 : 0) << 10)) << 13);
      S0.prv()[M + v] = M + v;
    }
  }
  __syncthreads();

  // ---- prologue 3: initial schedule (caller's CSR, or Algorithm 1 on the device)
  if (status == ASCHED_OK) {
    if (P.init_off) {
      int csr_bad = 0;
      for (int v = tid; v < V; v += nthr) {
        const int o0 = gin(P.init_off + v), o1 = gin(P.init_off + v + 1);
        if (o0 < 0 || o1 < o0 || o1 > M || (v == 0 && o0 != 0) || (v == V - 1 && o1 != M)) {
          csr_bad = 1;
          continue;
        }
        int prev = M + v;
        const int vw = nv_vw(S0.nv(M + v));
        for (int k = o0; k < o1; ++k) {
          const int m = gin(P.init_route + k);
          if (m < 0 || m >= M) {
            csr_bad = 1;
            break;
          }
          atomicAdd(&sm.cnt[m], 1);
          S0.nv(prev) = (S0.nv(prev) & ~kNodeMask) | m;
          S0.prv()[m] = prev;
          S0.nv(m) = (vw | ((P.heli_only ? gin(P.heli_only + m) : 0) << 11)) << 13;
          prev = m;
        }
        S0.nv(prev) = (S0.nv(prev) & ~kNodeMask) | (M + v);
        S0.prv()[M + v] = prev;
      }
      csr_bad = __syncthreads_or(csr_bad);
      if (!csr_bad) {
        int dup = 0;
        for (int m = tid; m < M; m += nthr) dup |= sm.cnt[m] != 1;
        csr_bad = __syncthreads_or(dup);
      }
      if (csr_bad) status = ASCHED_E_INVALID;
    } else {
      // Mission order: heli-only first, then by deadline, then by id.
      for (int m = tid; m < M; m += nthr) {
        const int hm = (P.heli_only && gin(P.heli_only + m)) ? 0 : 1, wmv = DL ? sm.wm[m] : 0;
        int r = 0;
        for (int k = 0; k < M; ++k) {
          const int hk = (P.heli_only && gin(P.heli_only + k)) ? 0 : 1, wk = DL ? sm.wm[k] : 0;
          r += (hk < hm) || (hk == hm && (wk < wmv || (wk == wmv && k < m)));
        }
        sm.order[r] = m;
      }
      __syncthreads();
      if (warp == 0) {
        for (int v = lane; v < V; v += 32) {
          sm.glast[v] = M + v;
          sm.gend[v] = sm.eloc[M + v];
          sm.gdep[v] = 0;
          sm.gfl[v] = 0;
        }
        __syncwarp();
        int fail = 0;
        for (int k = 0; k < M && !fail; ++k) {
          const int m = sm.order[k];
          const int w = sm.wm[m];
          const int heli = P.heli_only ? gin(P.heli_only + m) : 0;
          uint64_t best = kNoKey;
          for (int v = lane; v < V; v += 32) {
            const int tyl = sm.tyl[v];
            const int bl = sm.eloc[M + v];
            const int a = tb.a(tb.row(tyl, sm.gend[v]), m);
            const int bret = tb.b(tb.row(tyl, bl), m);
            const int last = sm.glast[v];
            const int old = last == M + v ? 0 : tb.b(tb.row(tyl, bl), last);
            const int app = a + bret - old;
            const int f = sm.gfl[v];
            bool ok = !(heli && sm.vtype[v] != 0);
            if (DL) ok = ok && (sm.gdep[v] + a <= w) && (w + bret <= c.horizon);
            int score;
            if (PEN) {
              score = app + c.lam * (pos0(f + app - c.cap) - pos0(f - c.cap));
            } else {
              ok = ok && (f + app <= c.cap);
              score = app;
            }
            if (ok) best = min_u64(best, pack_key(score, static_cast<uint32_t>(v)));
          }
          best = warp_min_key(best);
          if (best == kNoKey) {
            fail = 1;
            break;
          }
          if (lane == 0) {
            const int v = static_cast<int>(static_cast<uint32_t>(best));
            const int tyl = sm.tyl[v];
            const int bl = sm.eloc[M + v];
            const int last = sm.glast[v];
            const int a = tb.a(tb.row(tyl, sm.gend[v]), m);
            const int bret = tb.b(tb.row(tyl, bl), m);
            const int old = last == M + v ? 0 : tb.b(tb.row(tyl, bl), last);
            S0.nv(last) = (S0.nv(last) & ~kNodeMask) | m;
            S0.prv()[m] = last;
            S0.nv(m) = (M + v) | ((nv_vw(S0.nv(M + v)) | (heli << 11)) << 13);
            S0.prv()[M + v] = m;
            sm.glast[v] = m;
            sm.gend[v] = sm.eloc[m];
            sm.gdep[v] = w;
            sm.gfl[v] += a + bret - old;
          }
          __syncwarp();
        }
        if (lane == 0) sm.misc[MISC_GREEDY_FAIL] = fail;
      }
      __syncthreads();
      if (sm.misc[MISC_GREEDY_FAIL]) status = ASCHED_E_INFEASIBLE_INIT;
    }
  }

  // ---- prologue 4: flights, records, initial objective and feasibility
  int Z = 0;
  if (status == ASCHED_OK) {
    const Arr fl0 = sm.gfl;  // flight sums (greedy scratch is free now)
    __syncthreads();
    for (int v = tid; v < V; v += nthr) fl0[v] = 0;
    __syncthreads();
    for (int t = tid; t < N; t += nthr) {
      const int pv = S0.prv()[t];
      const int vw = nv_vw(S0.nv(t));
      const int tyl = vw_plane(vw) * L;
      int contrib;
      if (t < M) contrib = tb.a(tb.row(tyl, sm.eloc[pv]), t);
      else contrib = pv == t ? 0 : tb.b(tb.row(tyl, sm.sloc[t]), pv);
      atomicAdd(&fl0[vw_veh(vw)], contrib);
    }
    __syncthreads();
    int infeasible = 0;
    for (int t = tid; t < N; t += nthr) {
      const int nv = S0.nv(t), pv = S0.prv()[t];
      const int vw = nv_vw(nv);
      const int f = fl0[vw_veh(vw)];
      const int tyl = vw_plane(vw) * L;
      write_records<PEN, DL, BIG, RP>(sm, tb, S0, c, t, nv_next(nv), pv, vw, f);
      if (t < M) {
        infeasible |= (vw >> 11) & (vw >> 10) & 1;
        if (DL) {
          const int dep = pv < M ? sm.wm[pv] : 0;
          infeasible |= dep + tb.a(tb.row(tyl, sm.eloc[pv]), t) > sm.wm[t];
        }
      } else {
        if (!PEN) infeasible |= f > c.cap;
        if (DL && pv != t) infeasible |= sm.wm[pv] + tb.b(tb.row(tyl, sm.sloc[t]), pv) > c.horizon;
      }
    }
    if (__syncthreads_or(infeasible)) status = ASCHED_E_INFEASIBLE_INIT;
    if (warp == 0) {
      int z = 0;
      for (int v = lane; v < V; v += 32) {
        const int f = fl0[v];
        z += f + (PEN ? c.lam * pos0(f - c.cap) : 0);
      }
      z = __reduce_add_sync(0xffffffffu, z);
      if (lane == 0) sm.misc[MISC_Z0] = z;
    }
    for (int t = tid; t < N; t += nthr) sm.best[t] = nv_next(S0.nv(t));
    for (int i = tid; i < 2 * kMaxCluster; i += nthr) sm.slots()[i] = 0;
    if (tid < 2) sm.gkey()[tid] = 0;
    __syncthreads();
    Z = sm.misc[MISC_Z0];
  }

  // ---- main loop
  int zbest = Z, best_it = -1, it = 0;
  const bool looped = status == ASCHED_OK;  // uniform over the cluster
  if (looped) {
    if (C > 1) cluster_sync_all();
    // Static assignment over the item list [relocation pairs (N * ceil(M/2)) | swaps
    // (M(M-1)/2) | neighbour swaps (M, with RP records only)]: chunks of 32 consecutive items go round-robin to
    // (CTA, warp) over the K * C CTAs of the grid, so every CTA gets an equal share and
    // the lanes of a warp take consecutive items.
    // A relocation item i is (y, h) = divmod(i, H) for missions 2h and 2h + 1 (with RP
    // records for missions 4h .. 4h + 3); a swap
    // item j is (row, a) = divmod(j, M) with b = (a + row + 1) mod M, which lists every
    // pair a != b once (with RP records the pairs that are neighbours in a route are
    // masked there, and a neighbour item t swaps mission t with its successor when that
    // is a mission).
    // Coordinates advance by G without dividing.
    const int CT = K * C;
    const int G = CT * nthr;
    const int g = lane + 32 * (cid * C + rank + CT * warp);
    const int H = RP ? (M + 3) / 4 : (M + 1) / 2;  // relocation items per node y
    const int Rn = N * H;
    const int Sn = M * (M - 1) / 2;
    int r_y = N, r_h = 0, s_j = Sn, s_row = 0, s_a = 0, Gq = 0, Gr = 0, Sq = 0, Sr = 0, n_k = M;
    if (M > 0) {
      Gq = G / H;
      Gr = G - Gq * H;
      Sq = G / M;
      Sr = G - Sq * M;
      if (g < Rn) {
        r_y = g / H;
        r_h = g - r_y * H;
      }
      const int k = g < Rn ? (Rn - g + G - 1) / G : 0;  // relocation items of this thread
      s_j = g + k * G - Rn;
      if (s_j < Sn) {
        s_row = s_j / M;
        s_a = s_j - s_row * M;
      }
      const int k2 = g < Rn + Sn ? (Rn + Sn - g + G - 1) / G : 0;  // items before the neighbour pass
      n_k = g + k2 * G - (Rn + Sn);
    }
    const ItemCursor cursor{r_y, r_h, s_j, s_row, s_a, Gq, Gr, Sq, Sr, G, H, Sn, n_k};
    const int iters = DEBUG ? 1 : P.iterations;
    for (it = 0; it < iters; ++it) {
      const State S = S0;
      const int it_eval = DEBUG ? P.dbg_it : it;
      const int zb_eval = DEBUG ? P.dbg_zbest : zbest;
      // z_best - Z, clamped to int32 (a caller's z_best is arbitrary in DEBUG mode; every
      // delta lies well inside the int32 range, so the clamp changes no comparison)
      const int64_t zr = static_cast<int64_t>(zb_eval) - Z;
      const int zrel = static_cast<int>(zr < INT32_MIN ? INT32_MIN : (zr > INT32_MAX ? INT32_MAX : zr));
      uint64_t key = c.heli ? eval_items<PEN, DL, DEBUG, BIG, RP, true>(sm, tb, S, c, cursor, it_eval, zrel, P)
                            : eval_items<PEN, DL, DEBUG, BIG, RP, false>(sm, tb, S, c, cursor, it_eval, zrel, P);
      key = warp_min_key(key);
      if (lane == 0) sm.warpkey()[warp] = key;
      __syncthreads();
      uint64_t gk = warp_min_key(lane < nwarps ? sm.warpkey()[lane] : kNoKey);
      bool timed_out = false;
      if (C > 1) {
        // Push this CTA's key, tagged with the iteration, into slot [it & 1][rank] of
        // every CTA; then every warp polls its own C slots until all carry this
        // iteration's tag (bounded by the timeout).
        const int sb = it & 1;
        const uint64_t tag = iter_tag(it);
        const bool withhold = P.test_withhold && K == 1 && it == 0 && rank == C - 1;  // test hook
        if (warp == 0 && lane < C && !withhold) {
          const uint32_t slot_addr = smem_u32(&sm.slots()[sb * kMaxCluster + rank]);
          st_peer_u64(mapa_rank(slot_addr, lane), (gk & ~kTagMask) | tag);
        }
        const uint32_t my_slot = smem_u32(&sm.slots()[sb * kMaxCluster + (lane < C ? lane : 0)]);
        uint64_t v = ld_own_u64(my_slot);
        bool ok = __all_sync(0xffffffffu, (v & kTagMask) == tag);
        if (!ok) {
          const uint64_t t0 = global_ns();
          while (true) {
            v = ld_own_u64(my_slot);
            ok = __all_sync(0xffffffffu, (v & kTagMask) == tag);
            if (ok) break;
            // warp-uniform decision: lane 0's clock decides for the warp
            const bool late = __shfl_sync(0xffffffffu, (int64_t)(global_ns() - t0) > P.timeout_ns, 0);
            if (late) break;
          }
        }
        if (!ok) {
          timed_out = true;
        } else {
          gk = warp_min_key(lane < C ? v : kNoKey) & ~kTagMask;
          if ((gk >> 32) == 0xFFFFFFFFull) gk = kNoKey;  // real deltas never reach 2^31 - 1
        }
      }
      if (K > 1) {
        // Between clusters: rank 0 of each cluster stores the cluster's key, tagged, into
        // global slot [it & 1][cid]; warp 0 of every CTA polls the K slots until all carry
        // this iteration's tag (bounded), takes the least and stores it, tagged, into its
        // own CTA's shared memory, where every warp polls it. A wait that gives up is
        // stored as a key with kFailBit. (Every CTA polling L2 itself measured faster than
        // rank 0 polling and pushing the key to its peers over DSMEM; more polling warps
        // per CTA, or every CTA publishing its own key, slower.) The slots were zeroed
        // before the launch; a slot buffer is reused two iterations later, when every CTA
        // has read it (a cluster publishes for it + 1 only after its CTAs have read all
        // keys of it, the cluster exchange of it + 1 coming first).
        const int sb = it & 1;
        const uint64_t tag = iter_tag(it);
        const uint32_t gk_addr = smem_u32(&sm.gkey()[sb]);
        if (warp == 0) {
          uint64_t* gs = P.gslots + static_cast<int64_t>(sb) * P.gslot_stride;
          const bool withhold = P.test_withhold && it == 0 && cid == K - 1;  // test hook
          if (rank == 0 && lane == 0 && !timed_out && !withhold)
            st_relaxed_gpu_u64(gs + cid, (gk & ~(kTagMask | kFailBit)) | tag);
          bool ok = !timed_out;
          uint64_t m = kNoKey;
          if (ok) {
            const uint64_t t0 = global_ns();
            while (true) {
              bool mine = true;
              uint64_t mk = kNoKey;
              for (int k = lane; k < K; k += 32) {
                const uint64_t v = ld_relaxed_gpu_u64(gs + k);
                mine = mine && (v & kTagMask) == tag;
                mk = min_u64(mk, v);
              }
              if (__all_sync(0xffffffffu, mine)) {
                m = warp_min_key(mk);
                break;
              }
              if (__shfl_sync(0xffffffffu, static_cast<int64_t>(global_ns() - t0) > P.timeout_ns, 0)) {
                ok = false;
                break;
              }
            }
          }
          const uint64_t msg = ok ? ((m & ~kTagMask) | tag) : ((0xFFFFFFFFull << 32) | kFailBit | tag);
          if (lane == 0) st_own_u64(gk_addr, msg);
        }
        if (!timed_out) {
          uint64_t v = ld_own_u64(gk_addr);
          bool got = __all_sync(0xffffffffu, (v & kTagMask) == tag);
          if (!got) {
            const uint64_t t0 = global_ns();
            while (true) {
              v = ld_own_u64(gk_addr);
              got = __all_sync(0xffffffffu, (v & kTagMask) == tag);
              if (got) break;
              if (__shfl_sync(0xffffffffu, static_cast<int64_t>(global_ns() - t0) > P.timeout_ns, 0)) break;
            }
          }
          if (!got || (v & kFailBit)) {
            timed_out = true;
          } else {
            gk = v & ~kTagMask;
            if ((gk >> 32) == 0xFFFFFFFFull) gk = kNoKey;
          }
        }
      }
      // A chosen move must name nodes of this instance; anything else ends the solve
      // (gk is the same in every thread of the grid, so this decision is too).
      bool bad_key = false;
      if (!timed_out && gk != kNoKey) {
        const uint32_t id = static_cast<uint32_t>(gk);
        if (id & kSwapBit) {
          const uint32_t a = (id >> kIdShift) & kIdMask, b = id & kIdMask;
          bad_key = !(a < b && b < static_cast<uint32_t>(M));
        } else {
          const uint32_t m = id >> kIdShift, y = id & kIdMask;
          bad_key = !(m < static_cast<uint32_t>(M) && y < static_cast<uint32_t>(N) && y != m);
        }
      }
      if (DEBUG) {
        if (lead && tid == 0 && !timed_out) *P.dbg_key = gk;
      } else if (!timed_out && !bad_key && gk != kNoKey) {
        // ---- apply the chosen move, in place. A node's records depend only on its own
        // links, vehicle and route flight, and static tables: every thread first reads
        // the move's records (the decode and the two routes' new flights), then, after
        // one barrier, rewrites the nodes of the one or two changed routes (vehicles va,
        // vb), each thread its own nodes.
        const int Znew = Z + key_delta(gk);
        const bool improved = Znew < zbest;
        const uint32_t id = static_cast<uint32_t>(gk);
        const bool is_swap = (id & kSwapBit) != 0;
        // the move's nodes and links (relocation: m = n1 before y = n2; swap: a = n1, b = n2)
        const int n1 = static_cast<int>(is_swap ? ((id >> kIdShift) & kIdMask) : (id >> kIdShift));
        const int n2 = static_cast<int>(id & kIdMask);
        const int nv1 = S.nv(n1), nv2 = S.nv(n2);
        const int p1 = S.prv()[n1], p2 = S.prv()[n2];
        const int vwa = nv_vw(nv1), vwb = nv_vw(nv2);
        const int va = vw_veh(vwa), vb = vw_veh(vwb);
        const int x1 = nv_next(nv1), x2 = nv_next(nv2);
        const bool adjA = is_swap && x1 == n2;  // a immediately before b
        const bool adjB = is_swap && x2 == n1;  // b immediately before a
        const int f_src = moved_flight<BIG>(sm, tb, S, c, id, true);
        const int f_dst = moved_flight<BIG>(sm, tb, S, c, id, false);
        __syncthreads();  // no record is rewritten before every thread has read the move's
        for (int t = tid; t < N; t += nthr) {
          const int nv = S.nv(t);
          const int vt = nv_veh(nv);
          int nx = nv_next(nv);
          if (vt == va || vt == vb) {
            int pv = S.prv()[t], vw = nv_vw(nv);
            if (!is_swap) {  // e -> m -> s ... x -> y  becomes  e -> s ... x -> m -> y
              const int m = n1, y = n2, e = p1, sx = x1, x = p2;
              if (t == e) nx = sx;
              if (t == sx) pv = e;
              if (t == x) nx = m;
              if (t == y) pv = m;
              if (t == m) {
                nx = y;
                pv = x;
                vw = vw_move(vwb, vw);
              }
            } else {
              const int a = n1, b = n2, pa = p1, na = x1, pb = p2, nb = x2;
              if (adjA) {  // pa -> a -> b -> nb  becomes  pa -> b -> a -> nb
                if (t == pa) nx = b;
                if (t == nb) pv = a;
                if (t == b) {
                  pv = pa;
                  nx = a;
                }
                if (t == a) {
                  pv = b;
                  nx = nb;
                }
              } else if (adjB) {  // pb -> b -> a -> na  becomes  pb -> a -> b -> na
                if (t == pb) nx = a;
                if (t == na) pv = b;
                if (t == a) {
                  pv = pb;
                  nx = b;
                }
                if (t == b) {
                  pv = a;
                  nx = na;
                }
              } else {
                if (t == pa) nx = b;
                if (t == na) pv = b;
                if (t == pb) nx = a;
                if (t == nb) pv = a;
                if (t == a) {
                  pv = pb;
                  nx = nb;
                  vw = vw_move(vwb, vwa);
                }
                if (t == b) {
                  pv = pa;
                  nx = na;
                  vw = vw_move(vwa, vwb);
                }
              }
            }
            // The new flight of t's route is needed by route ends (FB) and, with RP
            // records, by every mission.
            const int f2 = vw_veh(vw) == va ? f_src : f_dst;
            write_records<PEN, DL, BIG, RP>(sm, tb, S, c, t, nx, pv, vw, f2);
          }
          if (improved) sm.best[t] = nx;
        }
        if (tid == 0) {
          tb.set_tabu(va, n1, it + P.tenure);
          if (is_swap) tb.set_tabu(vb, n2, it + P.tenure);
        }
        Z = Znew;
        if (improved) {
          zbest = Znew;
          best_it = it;
        }
      }
      if (!DEBUG && lead && tid == 0 && !timed_out) {
        if (P.traj_move) P.traj_move[it] = gk == kNoKey ? kNullMove : static_cast<uint32_t>(gk);
        if (P.traj_z) P.traj_z[it] = Z;
      }
      if (__syncthreads_or(timed_out || bad_key)) {
        status = bad_key ? ASCHED_E_INVALID : ASCHED_E_TIMEOUT;
        break;
      }
    }
  }

  // ---- epilogue: best schedule in CSR form (the lead CTA writes every output)
  if (lead && !DEBUG && status == ASCHED_OK && P.out_off) {
    const Arr lens = sm.gfl;  // scratch reuse (V entries)
    int walk_bad = 0;
    for (int v = tid; v < V; v += nthr) {
      int n = 0, t = sm.best[M + v];
      while (t != M + v && n <= M) {
        if (t < 0 || t >= M) {
          walk_bad = 1;
          break;
        }
        ++n;
        t = sm.best[t];
      }
      lens[v] = n;
      walk_bad |= n > M;
    }
    walk_bad = __syncthreads_or(walk_bad);
    if (tid == 0 && !walk_bad) {
      int o = 0;
      for (int v = 0; v < V; ++v) {
        P.out_off[v] = o;
        o += lens[v];
      }
      P.out_off[V] = o;
      walk_bad = o != M;
      sm.misc[MISC_CSR_BAD] = walk_bad;
    }
    __syncthreads();
    if (sm.misc[MISC_CSR_BAD]) walk_bad = 1;
    if (!walk_bad) {
      for (int v = tid; v < V; v += nthr) {
        const int32_t* T = P.travel + static_cast<int64_t>(sm.vtype[v]) * L * L;
        const int bl = sm.eloc[M + v];
        int o = 0;
        for (int w = 0; w < v; ++w) o += lens[w];
        int f = 0, prevloc = bl, t = sm.best[M + v];
        while (t != M + v) {
          P.out_route[o++] = t;
          f += gin(T + prevloc * L + sm.sloc[t]) + gin(T + sm.sloc[t] * L + sm.eloc[t]);
          prevloc = sm.eloc[t];
          t = sm.best[t];
        }
        if (lens[v] > 0) f += gin(T + prevloc * L + bl);
        if (P.out_flight) P.out_flight[v] = f;
        if (P.out_over) P.out_over[v] = pos0(f - c.cap);
      }
    } else {
      status = ASCHED_E_INVALID;
    }
  }
  if (lead && tid == 0 && P.info) {
    P.info[ASCHED_INFO_STATUS] = status;
    P.info[ASCHED_INFO_Z_BEST] = zbest;
    P.info[ASCHED_INFO_BEST_IT] = best_it;
    P.info[ASCHED_INFO_Z_INIT] = sm.misc[MISC_Z0];
    P.info[ASCHED_INFO_Z_FINAL] = Z;
    P.info[ASCHED_INFO_ITERS] = it;
    P.info[6] = 0;
    P.info[7] = 0;
  }
  // No CTA may leave while a peer can still write into its shared memory.
  if (C > 1 && looped) cluster_sync_unaligned();
}

template <bool PEN, bool DL, bool DEBUG, bool BIG>
__global__ void __launch_bounds__(kMaxThreads, 1) tabu_kernel(const __grid_constant__ KParams P) {
  const int C = P.cluster;
  const int K = P.grid_clusters > 1 ? P.grid_clusters : 1;
  if (!launch_shape_ok(C, K * C)) {  // uniform over the launch: every CTA returns here
    if (blockIdx.x == 0 && threadIdx.x == 0 && P.info) P.info[ASCHED_INFO_STATUS] = ASCHED_E_INVALID;
    return;
  }
  const int rank = C > 1 ? static_cast<int>(cluster_rank()) : 0;
  const int cid = K > 1 ? static_cast<int>(blockIdx.x) / C : 0;
  solve_one<PEN, DL, DEBUG, BIG, false>(P, P.lay, C, rank, K, cid);
}

// ------------------------------------------------------------------ batches --------

// Many instances in one launch. Instance b's arrays start at its offsets in the
// concatenated inputs; outputs are concatenated the same way. work[0] is a queue
// ticket counter (zeroed by batch_order_kernel), work[1 + k] the k-th instance to
// solve (largest first).
struct BParams {
  KParams run;  // tenure, iterations, lambda, nt, timeout; no instance pointers
  int32_t B;
  int32_t smem_words;  // dynamic shared memory of the launch
  int32_t compact;     // always take the int16 matrix layout
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
  int32_t* work;
};

__host__ __device__ inline int64_t moves_of(int64_t M, int64_t V) { return M * (M + V - 2) + M * (M - 1) / 2; }

// Processing order: instances by decreasing neighbourhood size (ties by index), so the
// persistent CTAs start the longest solves first. Also resets the ticket counter.
__global__ void batch_order_kernel(int32_t B, const int32_t* veh_off, const int32_t* mis_off, int32_t* work) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    const int64_t nb = moves_of(mis_off[b + 1] - mis_off[b], veh_off[b + 1] - veh_off[b]);
    int r = 0;
    for (int k = 0; k < B; ++k) {
      const int64_t nk = moves_of(mis_off[k + 1] - mis_off[k], veh_off[k + 1] - veh_off[k]);
      r += (nk > nb) || (nk == nb && k < b);
    }
    work[1 + r] = b;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) work[0] = 0;
}

// CL: the launch is made of thread-block clusters of Q.run.cluster CTAs and each instance
// is solved by a whole cluster (the same search as asched_solve with that cluster size):
// rank 0 takes the ticket and the other CTAs read it from rank 0's shared memory between
// two cluster barriers.
template <bool PEN, bool DL, bool CL>
__global__ void __launch_bounds__(kMaxThreads, 1) tabu_batch_kernel(const __grid_constant__ BParams Q) {
  __shared__ int s_ticket;
  const int C = CL ? Q.run.cluster : 1;
  if (CL && !launch_shape_ok(C, 0)) {  // uniform over the launch: nothing is solved
    if (blockIdx.x == 0)
      for (int b = threadIdx.x; b < Q.B; b += blockDim.x)
        Q.info[static_cast<int64_t>(b) * ASCHED_INFO_LEN + ASCHED_INFO_STATUS] = ASCHED_E_INVALID;
    return;
  }
  const int rank = CL ? static_cast<int>(cluster_rank()) : 0;
  while (true) {
    if (rank == 0 && threadIdx.x == 0) s_ticket = atomicAdd(&Q.work[0], 1);
    int k;
    if (CL) {
      cluster_sync_unaligned();  // thread 0 of rank 0 arrives from its claim
      k = rank == 0 ? s_ticket : ld_peer_i32(mapa_rank(smem_u32(&s_ticket), 0));
      cluster_sync_unaligned();  // every CTA has read it before rank 0 takes the next
    } else {
      __syncthreads();
      k = s_ticket;
      __syncthreads();
    }
    if (k >= Q.B) break;
    const int b = Q.work[1 + k];
    KParams P = Q.run;
    const int lo = Q.loc_off[b], vo = Q.veh_off[b], mo = Q.mis_off[b];
    P.L = Q.loc_off[b + 1] - lo;
    P.V = Q.veh_off[b + 1] - vo;
    P.M = Q.mis_off[b + 1] - mo;
    P.travel = Q.travel + Q.travel_off[b];
    P.veh_base = Q.veh_base + vo;
    P.veh_type = Q.veh_type ? Q.veh_type + vo : nullptr;
    P.pickup = Q.pickup + mo;
    P.delivery = Q.delivery + mo;
    P.heli_only = Q.heli_only ? Q.heli_only + mo : nullptr;
    P.deadline = Q.deadline ? Q.deadline + mo : nullptr;
    P.cap = Q.duty_cap[b];
    P.horizon = Q.horizon[b];
    P.out_off = Q.out_off + vo + b;
    P.out_route = Q.out_route + mo;
    P.out_flight = Q.out_flight + vo;
    P.out_over = Q.out_over + vo;
    P.info = Q.info + static_cast<int64_t>(b) * ASCHED_INFO_LEN;
    // Each instance takes the gather tables when they fit the launch's shared
    // memory, the int16 matrix otherwise.
    const Layout small = make_layout(P.M, P.V, P.L, P.nt, false, true);
    if (!Q.compact && small.total <= Q.smem_words) {
      solve_one<PEN, DL, false, false, true>(P, small, C, rank, 1, 0);
    } else {
      const Layout big = make_layout(P.M, P.V, P.L, P.nt, true, true);
      solve_one<PEN, DL, false, true, true>(P, big, C, rank, 1, 0);
    }
    __syncthreads();  // the next instance's prologue reuses shared memory
  }
}

// ------------------------------------------------------------------ serving --------

// A persistent launch that serves requests as the host publishes them. Each request
// sits in a fixed-capacity slot (inputs) with a matching output slot; the host writes
// a slot, appends its index to the ring and raises control[PUBLISHED], all by copies
// ordered on one stream. A CTA takes the next ticket, solves that slot's instance with
// the same per-instance search as asched_solve, and writes the request's sequence
// number to done[slot]. Every wait is bounded: the launch ends when control[STOP] is
// set and every published ticket is taken, or after idle_ns without a new ticket.
struct SParams {
  KParams run;
  int32_t n_slots, ring_len, Lc, Vc, Mc, nt;
  int32_t slot_words, out_words, smem_words, compact;
  int64_t idle_ns;
  const int32_t* slot_data;
  int32_t* slot_out;
  const int32_t* ring;
  int32_t* control;
  int32_t* done;
};

__host__ __device__ inline int serve_slot_words(int Lc, int Vc, int Mc, int nt) {
  return round_up(ASCHED_SLOT_HEADER + nt * Lc * Lc + 2 * Vc + 4 * Mc, 4);
}
__host__ __device__ inline int serve_out_words(int Vc, int Mc) {
  return round_up(3 * Vc + 1 + Mc + ASCHED_INFO_LEN, 4);
}

__device__ __forceinline__ int ld_volatile_i32(const int32_t* p) { return *reinterpret_cast<const volatile int32_t*>(p); }

// CL: the launch is made of thread-block clusters of Q.run.cluster CTAs and each request
// is solved by a whole cluster (the same search as asched_solve with that cluster size):
// rank 0 claims the ticket and the others read it from rank 0's shared memory between
// two cluster barriers. Their wait at the barrier ends when rank 0 arrives, which its own
// bounded claim loop guarantees.
template <bool PEN, bool DL, bool CL>
__global__ void __launch_bounds__(kMaxThreads, 1) serve_kernel(const __grid_constant__ SParams Q) {
  __shared__ int s_ticket;
  const int C = CL ? Q.run.cluster : 1;
  if (CL && !launch_shape_ok(C, 0)) return;  // uniform over the launch; nothing is served
  const int rank = CL ? static_cast<int>(cluster_rank()) : 0;
  if (threadIdx.x == 0) atomicAdd(&Q.control[ASCHED_CTRL_STARTED], 1);
  uint64_t idle_since = global_ns();
  while (true) {
    if (rank == 0 && threadIdx.x == 0) {
      int got;
      while (true) {
        const int pub = ld_volatile_i32(&Q.control[ASCHED_CTRL_PUBLISHED]);
        const int cl = ld_volatile_i32(&Q.control[ASCHED_CTRL_CLAIMED]);
        if (cl < pub) {
          if (atomicCAS(&Q.control[ASCHED_CTRL_CLAIMED], cl, cl + 1) == cl) {
            got = cl;
            break;
          }
          continue;
        }
        if (ld_volatile_i32(&Q.control[ASCHED_CTRL_STOP])) {
          got = -1;
          break;
        }
        if (static_cast<int64_t>(global_ns() - idle_since) > Q.idle_ns) {
          atomicAdd(&Q.control[ASCHED_CTRL_IDLE_EXITS], 1);
          got = -1;
          break;
        }
        __nanosleep(1000);
      }
      s_ticket = got;
    }
    int t;
    if (CL) {
      cluster_sync_unaligned();  // thread 0 of rank 0 arrives from its claim loop
      t = rank == 0 ? s_ticket : ld_peer_i32(mapa_rank(smem_u32(&s_ticket), 0));
      cluster_sync_unaligned();  // every CTA has read it before rank 0 claims the next
    } else {
      __syncthreads();
      t = s_ticket;
      __syncthreads();
    }
    if (t < 0) break;
    const int slot = ld_volatile_i32(&Q.ring[t % Q.ring_len]);
    const int32_t* in = Q.slot_data + static_cast<int64_t>(slot) * Q.slot_words;
    int32_t* out = Q.slot_out + static_cast<int64_t>(slot) * Q.out_words;
    const int L = gin(in), V = gin(in + 1), M = gin(in + 2);
    KParams P = Q.run;
    P.L = L;
    P.V = V;
    P.M = M;
    P.cap = gin(in + 3);
    P.horizon = gin(in + 4);
    const int flags = gin(in + 5);
    const int32_t* vb = in + ASCHED_SLOT_HEADER + Q.nt * Q.Lc * Q.Lc;
    P.travel = in + ASCHED_SLOT_HEADER;
    P.veh_base = vb;
    P.veh_type = vb + Q.Vc;
    P.pickup = vb + 2 * Q.Vc;
    P.delivery = P.pickup + Q.Mc;
    P.heli_only = (flags & 1) ? P.delivery + Q.Mc : nullptr;
    P.deadline = (flags & 2) ? P.delivery + 2 * Q.Mc : nullptr;
    P.out_off = out;
    P.out_route = out + Q.Vc + 1;
    P.out_flight = P.out_route + Q.Mc;
    P.out_over = P.out_flight + Q.Vc;
    P.info = P.out_over + Q.Vc;
    const bool sizes_ok = L >= 1 && L <= Q.Lc && V >= 1 && V <= Q.Vc && M >= 0 && M <= Q.Mc &&
                          (DL == ((flags & 2) != 0));
    if (sizes_ok) {
      const Layout small = make_layout(M, V, L, Q.nt, false, true);
      if (!Q.compact && small.total <= Q.smem_words) {
        solve_one<PEN, DL, false, false, true>(P, small, C, rank, 1, 0);
      } else {
        const Layout big = make_layout(M, V, L, Q.nt, true, true);
        if (big.total <= Q.smem_words) {
          solve_one<PEN, DL, false, true, true>(P, big, C, rank, 1, 0);
        } else if (rank == 0 && threadIdx.x == 0) {
          P.info[ASCHED_INFO_STATUS] = ASCHED_E_TOO_LARGE;
        }
      }
    } else if (rank == 0 && threadIdx.x == 0) {
      P.info[ASCHED_INFO_STATUS] = ASCHED_E_INVALID;
    }
    __syncthreads();
    if (rank == 0 && threadIdx.x == 0) {
      __threadfence_system();
      *reinterpret_cast<volatile int32_t*>(&Q.done[slot]) = gin(in + 6);
      atomicAdd(&Q.control[ASCHED_CTRL_SERVED], 1);
    }
    idle_since = global_ns();
  }
}

// ------------------------------------------------------------------ host side ------

template <bool PEN, bool DL, bool DEBUG, bool BIG>
void* kernel_ptr() {
  return reinterpret_cast<void*>(&tabu_kernel<PEN, DL, DEBUG, BIG>);
}

template <bool DEBUG, bool BIG>
void* pick_kernel_b(bool pen, bool dl) {
  if (pen) return dl ? kernel_ptr<true, true, DEBUG, BIG>() : kernel_ptr<true, false, DEBUG, BIG>();
  return dl ? kernel_ptr<false, true, DEBUG, BIG>() : kernel_ptr<false, false, DEBUG, BIG>();
}

void* pick_kernel(bool pen, bool dl, bool debug, bool big) {
  if (debug) return big ? pick_kernel_b<true, true>(pen, dl) : pick_kernel_b<true, false>(pen, dl);
  return big ? pick_kernel_b<false, true>(pen, dl) : pick_kernel_b<false, false>(pen, dl);
}

// Shared-memory layout for an instance: the gather tables when they fit, else the
// int16 matrix (whose stamps limit iterations + tenure to 32,767). rp: the batch and
// serving kernels' layout, with the RP records.
int choose_layout(int M, int V, int L, int nt, const asched_params* p, int limit_bytes, bool rp, Layout* out) {
  const Layout small = make_layout(M, V, L, nt, false, rp);
  if (!(p->flags & ASCHED_COMPACT_LAYOUT) && static_cast<int64_t>(small.total) * 4 + 64 <= limit_bytes) {
    *out = small;
    return ASCHED_OK;
  }
  const Layout big = make_layout(M, V, L, nt, true, rp);
  if (static_cast<int64_t>(big.total) * 4 + 64 > limit_bytes) return ASCHED_E_TOO_LARGE;
  if (static_cast<int64_t>(p->iterations) + p->tenure > 32767) return ASCHED_E_TOO_LARGE;
  *out = big;
  return ASCHED_OK;
}

int check_sizes(const asched_instance* inst, const asched_params* p) {
  if (!inst || !p) return ASCHED_E_INVALID;
  if (inst->n_loc < 1 || inst->n_types < 1 || inst->n_types > 2) return ASCHED_E_INVALID;
  if (inst->n_vehicles < 1 || inst->n_missions < 0) return ASCHED_E_INVALID;
  if (inst->n_vehicles > kMaxVehicles || inst->n_missions > kMaxMissions ||
      inst->n_missions + inst->n_vehicles > kMaxNodes)
    return ASCHED_E_TOO_LARGE;
  if (inst->duty_cap < 0 || inst->horizon < 0) return ASCHED_E_INVALID;
  if (p->tenure < 0 || p->iterations < 0 || p->lambda < 0) return ASCHED_E_INVALID;
  if (p->cap_mode != ASCHED_HARD && p->cap_mode != ASCHED_PENALTY) return ASCHED_E_INVALID;
  if (p->cluster_size != 0 && p->cluster_size != 1 && p->cluster_size != 2 && p->cluster_size != 4 &&
      p->cluster_size != 8 && p->cluster_size != 16)
    return ASCHED_E_INVALID;
  if (p->block_threads != 0 && (p->block_threads < 64 || p->block_threads > kMaxThreads || p->block_threads % 32))
    return ASCHED_E_INVALID;
  if (p->timeout_ns < 0 || (p->flags & ~(ASCHED_COMPACT_LAYOUT | ASCHED_TEST_WITHHOLD_KEY | ASCHED_PLAIN_LAUNCH)) != 0)
    return ASCHED_E_INVALID;
  if (p->grid_clusters < 0 || p->grid_clusters > kMaxGridClusters) return ASCHED_E_INVALID;
  return ASCHED_OK;
}


int max_smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return -1;
  return v;
}

// Clusters of C CTAs (threads each, smem bytes of shared memory) that the device can
// hold at once for kernel fn; 0 when none fits.
int active_clusters(void* fn, int C, int threads, int smem, int* out) {
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return ASCHED_E_CUDA;
  if (C > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return ASCHED_E_CUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = static_cast<size_t>(smem);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    n = 0;
  }
  *out = n;
  return ASCHED_OK;
}

// Warps per CTA for a neighbourhood of `chunks` 32-item chunks dealt over `ctas` CTAs:
// the fewest, in steps of 4 (equal shares for an SM's four schedulers), that keep the
// largest per-warp share at its least (16 warps at most).
int warps_for(int64_t chunks, int64_t ctas) {
  const int64_t least = (chunks + 16 * ctas - 1) / (16 * ctas);
  int w = 4;
  while (w < 16 && (chunks + w * ctas - 1) / (w * ctas) > least) w += 4;
  return w;
}

// Bytes of the global key slots a launch of K clusters uses: two buffers of K keys,
// each buffer in its own 128-byte lines.
int64_t grid_slot_stride(int K) { return round_up(K, 16); }  // in uint64 words
size_t grid_workspace_bytes(int K) { return K > 1 ? static_cast<size_t>(2 * grid_slot_stride(K) * 8) : 0; }

// Launch shape: block size, cluster size C and clusters K; returns status.
// allow_grid: the call has a workspace for the keys between clusters (K may exceed 1).
int make_plan(const asched_instance* inst, const asched_params* p, bool debug, bool allow_grid,
              asched_plan_t* plan, Layout* lay_out) {
  int rc = check_sizes(inst, p);
  if (rc != ASCHED_OK) return rc;
  if (p->grid_clusters < 0 || (!allow_grid && p->grid_clusters > 1)) return ASCHED_E_INVALID;
  const int M = inst->n_missions, V = inst->n_vehicles;
  const int limit = max_smem_optin();
  if (limit < 0) return ASCHED_E_CUDA;
  Layout lay;
  rc = choose_layout(M, V, inst->n_loc, inst->n_types, p, limit, false, &lay);
  if (rc != ASCHED_OK) return rc;
  const int bytes = lay.total * 4;
  void* fn = pick_kernel(p->cap_mode == ASCHED_PENALTY, inst->deadline != nullptr, debug, lay.big);
  const int64_t items = static_cast<int64_t>(M + V) * M + static_cast<int64_t>(M) * (M - 1) / 2;
  const int64_t evals = static_cast<int64_t>(M + V) * ((M + 1) / 2) + static_cast<int64_t>(M) * (M - 1) / 2;
  const int64_t chunks = (evals + 31) / 32;
  // Neighbourhoods of 1,024 items or more take the largest cluster. The evaluation deals
  // 32-item chunks of its item list (relocation pairs, then swaps) round-robin over the
  // warps of every CTA, so an iteration lasts as long as the warp with the most chunks,
  // plus a little per warp (reduce, decode, rewrite, barriers): such neighbourhoods take
  // the fewest warps per CTA that keep that largest share at its least (warps_for).
  // Measured on neighbourhoods of 1,778 to 259,800 moves, this was the fastest shape or
  // within 1 % of it. Smaller neighbourhoods take one thread per item and the fewest CTAs
  // that cover them.
  const bool wide = items >= 1024;
  int cl = p->cluster_size;
  if (cl == 0 && wide) cl = kMaxCluster;
  int K = p->grid_clusters > 0 ? p->grid_clusters : 1;
  const int probe_threads = p->block_threads ? p->block_threads : kMaxThreads;
  if (p->cluster_size == 0 && cl > 1) {
    // shrink the cluster until the device can place one
    int n = 0;
    while (cl > 1) {
      rc = active_clusters(fn, cl, probe_threads, bytes, &n);
      if (rc != ASCHED_OK) return rc;
      if (n > 0) break;
      cl /= 2;
    }
  }
  // Neighbourhoods with more than 4 chunks per warp on one full cluster (the evaluation
  // then dominates the iteration) spread over every cluster of that size the device
  // holds at once, when the call has a workspace. The largest cluster is kept: keys
  // cross clusters through L2, which costs about 2 us per iteration whatever the number
  // of clusters, so fewer, larger clusters (more of the exchange in DSMEM) measured
  // fastest (on the large instance 7 x 16 CTAs: 3.7 us per iteration; 15 x 8: 3.8;
  // 27 x 4: 4.1; 76 x 2: 5.2).
  if (allow_grid && p->grid_clusters == 0 && wide && chunks > 4 * 16 * static_cast<int64_t>(kMaxCluster)) {
    int n = 0;
    rc = active_clusters(fn, cl, probe_threads, bytes, &n);
    if (rc != ASCHED_OK) return rc;
    if (n >= 2) K = n;
  }
  if (cl == 0) cl = 1;
  int threads = p->block_threads;
  if (threads == 0) {
    if (wide) {
      threads = 32 * warps_for(chunks, static_cast<int64_t>(cl) * K);
    } else {
      const int64_t want = items > M + V ? items : M + V;
      threads = want >= kMaxThreads ? kMaxThreads : (want <= 64 ? 64 : round_up(static_cast<int>(want), 32));
    }
  }
  if (p->cluster_size == 0 && !wide && K == 1) {
    cl = 1;
    while (cl < kMaxCluster && items > static_cast<int64_t>(cl) * threads) cl *= 2;
    int n = 0;
    while (cl > 1) {  // shrink the cluster until the device can place one
      rc = active_clusters(fn, cl, threads, bytes, &n);
      if (rc != ASCHED_OK) return rc;
      if (n > 0) break;
      cl /= 2;
    }
  }
  if (K > 1) {  // every cluster must be resident at once
    int n = 0;
    rc = active_clusters(fn, cl, threads, bytes, &n);
    if (rc != ASCHED_OK) return rc;
    if (K > n) return ASCHED_E_TOO_LARGE;
  }
  plan->cluster_size = cl;
  plan->block_threads = threads;
  plan->smem_bytes = bytes;
  plan->moves_per_iteration = moves_of(M, V);
  plan->grid_clusters = K;
  plan->workspace_bytes = static_cast<int64_t>(grid_workspace_bytes(K));
  if (lay_out) *lay_out = lay;
  return ASCHED_OK;
}

int launch(const asched_instance* inst, const asched_params* p, bool debug, KParams kp, void* workspace,
           size_t ws_bytes, bool allow_grid, void* stream) {
  asched_plan_t plan;
  Layout lay;
  int rc = make_plan(inst, p, debug, allow_grid, &plan, &lay);
  if (rc != ASCHED_OK) return rc;
  if (!inst->travel || !inst->veh_base) return ASCHED_E_INVALID;
  if (inst->n_missions > 0 && (!inst->pickup || !inst->delivery)) return ASCHED_E_INVALID;
  const int K = plan.grid_clusters;
  if (K > 1 && (!workspace || ws_bytes < grid_workspace_bytes(K) || (reinterpret_cast<uintptr_t>(workspace) & 127u)))
    return ASCHED_E_INVALID;
  const bool pen = p->cap_mode == ASCHED_PENALTY;
  const bool dl = inst->deadline != nullptr;
  void* fn = pick_kernel(pen, dl, debug, lay.big);
  kp.travel = inst->travel;
  kp.veh_base = inst->veh_base;
  kp.veh_type = inst->veh_type;
  kp.pickup = inst->pickup;
  kp.delivery = inst->delivery;
  kp.heli_only = inst->heli_only;
  kp.deadline = inst->deadline;
  kp.L = inst->n_loc;
  kp.nt = inst->n_types;
  kp.V = inst->n_vehicles;
  kp.M = inst->n_missions;
  kp.cap = inst->duty_cap;
  kp.horizon = inst->horizon;
  kp.tenure = p->tenure;
  kp.iterations = p->iterations;
  kp.lambda = pen ? p->lambda : 0;
  kp.cluster = plan.cluster_size;
  kp.grid_clusters = K;
  kp.gslot_stride = static_cast<int32_t>(grid_slot_stride(K));
  kp.gslots = K > 1 ? static_cast<uint64_t*>(workspace) : nullptr;
  kp.timeout_ns = p->timeout_ns > 0 ? p->timeout_ns : kDefaultTimeoutNs;
  kp.test_withhold = (p->flags & ASCHED_TEST_WITHHOLD_KEY) ? 1 : 0;
  kp.lay = lay;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.smem_bytes) != cudaSuccess)
    return ASCHED_E_CUDA;
  if (plan.cluster_size > 8 &&
      cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return ASCHED_E_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (K > 1 && cudaMemsetAsync(workspace, 0, grid_workspace_bytes(K), st) != cudaSuccess) {
    (void)cudaGetLastError();
    return ASCHED_E_CUDA;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(plan.cluster_size * K, 1, 1);
  cfg.blockDim = dim3(plan.block_threads, 1, 1);
  cfg.dynamicSmemBytes = static_cast<size_t>(plan.smem_bytes);
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = plan.cluster_size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  // Clusters that wait on one another need to be resident together: a cooperative
  // launch guarantees it (or fails to launch).
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (K > 1 && !(p->flags & ASCHED_PLAIN_LAUNCH)) ? 2 : 1;
  void* args[] = {&kp};
  if (cudaLaunchKernelExC(&cfg, fn, args) != cudaSuccess) {
    (void)cudaGetLastError();
    return ASCHED_E_CUDA;
  }
  return ASCHED_OK;
}

template <bool PEN, bool DL, bool CL>
void* batch_kernel_ptr() {
  return reinterpret_cast<void*>(&tabu_batch_kernel<PEN, DL, CL>);
}

template <bool CL>
void* pick_batch_kernel(bool pen, bool dl) {
  return pen ? (dl ? batch_kernel_ptr<true, true, CL>() : batch_kernel_ptr<true, false, CL>())
             : (dl ? batch_kernel_ptr<false, true, CL>() : batch_kernel_ptr<false, false, CL>());
}

int launch_batch(const asched_batch* bt, const asched_params* p, const asched_batch_result* out,
                 void* workspace, size_t ws_bytes, void* stream) {
  if (!bt || !p || !out) return ASCHED_E_INVALID;
  const int B = bt->n_instances;
  if (B < 0) return ASCHED_E_INVALID;
  if (B == 0) return ASCHED_OK;
  if (!bt->h_loc_off || !bt->h_veh_off || !bt->h_mis_off || !bt->loc_off || !bt->veh_off || !bt->mis_off ||
      !bt->travel_off || !bt->travel || !bt->veh_base || !bt->pickup || !bt->delivery || !bt->duty_cap ||
      !bt->horizon)
    return ASCHED_E_INVALID;
  if (!out->route_off || !out->route || !out->info || !workspace) return ASCHED_E_INVALID;
  if (ws_bytes < sizeof(int32_t) * (static_cast<size_t>(B) + 1)) return ASCHED_E_INVALID;
  const int limit = max_smem_optin();
  if (limit < 0) return ASCHED_E_CUDA;
  int max_words = 0;
  asched_instance one = {};
  one.n_types = bt->n_types;
  one.duty_cap = 0;
  one.horizon = 0;
  for (int b = 0; b < B; ++b) {
    one.n_loc = bt->h_loc_off[b + 1] - bt->h_loc_off[b];
    one.n_vehicles = bt->h_veh_off[b + 1] - bt->h_veh_off[b];
    one.n_missions = bt->h_mis_off[b + 1] - bt->h_mis_off[b];
    int rc = check_sizes(&one, p);
    if (rc != ASCHED_OK) return rc;
    Layout lay;
    rc = choose_layout(one.n_missions, one.n_vehicles, one.n_loc, one.n_types, p, limit, true, &lay);
    if (rc != ASCHED_OK) return rc;
    if (lay.total > max_words) max_words = lay.total;
  }
  const int64_t bytes = static_cast<int64_t>(max_words) * 4;
  const bool pen = p->cap_mode == ASCHED_PENALTY;
  const bool dl = bt->deadline != nullptr;
  // CTAs per instance: 1 (one persistent CTA per SM slot) or a cluster of C CTAs
  const int C = p->cluster_size > 1 ? p->cluster_size : 1;
  void* fn = C > 1 ? pick_batch_kernel<true>(pen, dl) : pick_batch_kernel<false>(pen, dl);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)) !=
      cudaSuccess)
    return ASCHED_E_CUDA;
  const int threads = p->block_threads ? p->block_threads : kMaxThreads;
  int grid = 0;
  if (C > 1) {
    int n = 0;
    const int rc = active_clusters(fn, C, threads, static_cast<int>(bytes), &n);
    if (rc != ASCHED_OK) return rc;
    if (n < 1) return ASCHED_E_TOO_LARGE;
    grid = (B < n ? B : n) * C;
  } else {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, static_cast<size_t>(bytes)) !=
            cudaSuccess) {
      (void)cudaGetLastError();
      return ASCHED_E_CUDA;
    }
    if (per_sm < 1) return ASCHED_E_TOO_LARGE;
    grid = B < sms * per_sm ? B : sms * per_sm;
  }
  BParams q = {};
  q.run.nt = bt->n_types;
  q.run.tenure = p->tenure;
  q.run.iterations = p->iterations;
  q.run.lambda = pen ? p->lambda : 0;
  q.run.cluster = C;
  q.run.timeout_ns = p->timeout_ns > 0 ? p->timeout_ns : kDefaultTimeoutNs;
  q.B = B;
  q.smem_words = max_words;
  q.compact = (p->flags & ASCHED_COMPACT_LAYOUT) ? 1 : 0;
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
  q.work = static_cast<int32_t*>(workspace);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  batch_order_kernel<<<(B + 255) / 256, 256, 0, st>>>(B, bt->veh_off, bt->mis_off, q.work);
  if (cudaGetLastError() != cudaSuccess) return ASCHED_E_CUDA;
  void* args[] = {&q};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = static_cast<size_t>(bytes);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = C > 1 ? 1 : 0;
  if (cudaLaunchKernelExC(&cfg, fn, args) != cudaSuccess) {
    (void)cudaGetLastError();
    return ASCHED_E_CUDA;
  }
  return ASCHED_OK;
}

template <bool PEN, bool DL, bool CL>
void* serve_kernel_ptr() {
  return reinterpret_cast<void*>(&serve_kernel<PEN, DL, CL>);
}

template <bool CL>
void* pick_serve(bool pen, bool dl) {
  return pen ? (dl ? serve_kernel_ptr<true, true, CL>() : serve_kernel_ptr<true, false, CL>())
             : (dl ? serve_kernel_ptr<false, true, CL>() : serve_kernel_ptr<false, false, CL>());
}

// Load every serving kernel now. Kernels are loaded on first use, and loading one can
// wait for the device to go idle: a second persistent launch started while a first one
// runs (the cluster lane and the one-CTA lane of a server) would then wait until the
// first ends, which for a persistent launch is only its idle timeout.
int preload_serve_kernels() {
  void* fns[] = {pick_serve<false>(false, false), pick_serve<false>(false, true), pick_serve<false>(true, false),
                 pick_serve<false>(true, true),   pick_serve<true>(false, false),  pick_serve<true>(false, true),
                 pick_serve<true>(true, false),   pick_serve<true>(true, true)};
  for (void* fn : fns) {
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, fn) != cudaSuccess) {
      (void)cudaGetLastError();
      return ASCHED_E_CUDA;
    }
  }
  return ASCHED_OK;
}

int launch_serve(const asched_server* sv, const asched_params* p, int64_t idle_ns, int32_t max_ctas, void* stream) {
  if (!sv || !p) return ASCHED_E_INVALID;
  if (sv->n_slots < 1 || sv->ring_len < sv->n_slots || sv->max_loc < 1 || sv->max_vehicles < 1 ||
      sv->max_missions < 0 || sv->n_types < 1 || sv->n_types > 2 || idle_ns <= 0)
    return ASCHED_E_INVALID;
  if (!sv->slot_data || !sv->slot_out || !sv->ring || !sv->control || !sv->done) return ASCHED_E_INVALID;
  asched_instance cap = {};
  cap.n_loc = sv->max_loc;
  cap.n_types = sv->n_types;
  cap.n_vehicles = sv->max_vehicles;
  cap.n_missions = sv->max_missions;
  int rc = check_sizes(&cap, p);
  if (rc != ASCHED_OK) return rc;
  const int C = p->cluster_size > 1 ? p->cluster_size : 1;
  if (C > 1 && max_ctas > 0 && max_ctas < C) return ASCHED_E_INVALID;
  rc = preload_serve_kernels();
  if (rc != ASCHED_OK) return rc;
  const int limit = max_smem_optin();
  if (limit < 0) return ASCHED_E_CUDA;
  Layout lay;  // the largest request the slots can hold sizes the launch
  rc = choose_layout(sv->max_missions, sv->max_vehicles, sv->max_loc, sv->n_types, p, limit, true, &lay);
  if (rc != ASCHED_OK) return rc;
  const int64_t bytes = static_cast<int64_t>(lay.total) * 4;
  const bool pen = p->cap_mode == ASCHED_PENALTY;
  const bool dl = sv->has_deadlines != 0;
  void* fn = C > 1 ? pick_serve<true>(pen, dl) : pick_serve<false>(pen, dl);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)) !=
      cudaSuccess)
    return ASCHED_E_CUDA;
  if (C > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return ASCHED_E_CUDA;
  const int threads = p->block_threads ? p->block_threads : kMaxThreads;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return ASCHED_E_CUDA;
  }
  SParams q = {};
  q.run.nt = sv->n_types;
  q.run.tenure = p->tenure;
  q.run.iterations = p->iterations;
  q.run.lambda = pen ? p->lambda : 0;
  q.run.cluster = C;
  q.run.timeout_ns = p->timeout_ns > 0 ? p->timeout_ns : kDefaultTimeoutNs;
  q.n_slots = sv->n_slots;
  q.ring_len = sv->ring_len;
  q.Lc = sv->max_loc;
  q.Vc = sv->max_vehicles;
  q.Mc = sv->max_missions;
  q.nt = sv->n_types;
  q.slot_words = serve_slot_words(q.Lc, q.Vc, q.Mc, q.nt);
  q.out_words = serve_out_words(q.Vc, q.Mc);
  q.smem_words = lay.total;
  q.compact = (p->flags & ASCHED_COMPACT_LAYOUT) ? 1 : 0;
  q.idle_ns = idle_ns;
  q.slot_data = sv->slot_data;
  q.slot_out = sv->slot_out;
  q.ring = sv->ring;
  q.control = sv->control;
  q.done = sv->done;
  void* args[] = {&q};
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = static_cast<size_t>(bytes);
  cfg.stream = static_cast<cudaStream_t>(stream);
  cudaLaunchAttribute attr[1];
  int grid;
  if (C > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(C, 1, 1);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) != cudaSuccess) {
      (void)cudaGetLastError();
      return ASCHED_E_CUDA;
    }
    if (clusters < 1) return ASCHED_E_TOO_LARGE;
    int want = (max_ctas > 0 ? max_ctas : sms) / C;  // whole clusters only
    grid = C * (want < clusters ? want : clusters);
  } else {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, static_cast<size_t>(bytes)) !=
        cudaSuccess) {
      (void)cudaGetLastError();
      return ASCHED_E_CUDA;
    }
    if (per_sm < 1) return ASCHED_E_TOO_LARGE;
    grid = sms * per_sm;
    if (max_ctas > 0 && max_ctas < grid) grid = max_ctas;
  }
  cfg.gridDim = dim3(grid, 1, 1);
  if (cudaLaunchKernelExC(&cfg, fn, args) != cudaSuccess) {
    (void)cudaGetLastError();
    return ASCHED_E_CUDA;
  }
  return ASCHED_OK;
}

}  // namespace

// ------------------------------------------------------------------ fixed scratch ---

// Work queue and processing order for asched_solve_batch_static: a fixed array in
// every device's global memory, so that call needs no workspace from its caller.
// Host code only uses its device address, looked up on each call (see below).
static __device__ __align__(256) int32_t g_batch_scratch[1 + ASCHED_STATIC_BATCH_MAX];

namespace {

// Device address of g_batch_scratch on the current device. Looked up on every call
// (the lookup allocates nothing), so the address stays right after a device reset,
// which reloads the module and may move the array. The first lookup on a device can
// load the module, so it belongs before any stream capture.
int static_scratch(void** out) {
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_batch_scratch) != cudaSuccess || !ptr) {
    (void)cudaGetLastError();
    return ASCHED_E_CUDA;
  }
  *out = ptr;
  return ASCHED_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI ----------

extern "C" {

int asched_abi_version(void) { return ASCHED_ABI_VERSION; }

const char* asched_status_string(int status) {
  switch (status) {
    case ASCHED_OK: return "ok";
    case ASCHED_E_INVALID: return "invalid argument or instance data";
    case ASCHED_E_TOO_LARGE: return "instance too large for the on-chip layout";
    case ASCHED_E_OVERFLOW_GUARD: return "int32 objective could overflow";
    case ASCHED_E_INFEASIBLE_INIT: return "no feasible initial schedule";
    case ASCHED_E_TIMEOUT: return "a bounded device wait timed out";
    case ASCHED_E_CUDA: return "CUDA runtime error";
    default: return "unknown status";
  }
}

int asched_num_moves(int32_t n_missions, int32_t n_vehicles, int64_t* out) {
  if (!out || n_missions < 0 || n_vehicles < 1) return ASCHED_E_INVALID;
  *out = moves_of(n_missions, n_vehicles);
  return ASCHED_OK;
}

int asched_check_instance_host(const asched_instance* inst, const asched_params* p) {
  int rc = check_sizes(inst, p);
  if (rc != ASCHED_OK) return rc;
  const int L = inst->n_loc, V = inst->n_vehicles, M = inst->n_missions, nt = inst->n_types;
  if (!inst->travel || !inst->veh_base || (M > 0 && (!inst->pickup || !inst->delivery))) return ASCHED_E_INVALID;
  int64_t maxT = 0;
  for (int64_t i = 0; i < static_cast<int64_t>(nt) * L * L; ++i) {
    if (inst->travel[i] < 0) return ASCHED_E_INVALID;
    if (inst->travel[i] > maxT) maxT = inst->travel[i];
  }
  for (int v = 0; v < V; ++v) {
    if (inst->veh_base[v] < 0 || inst->veh_base[v] >= L) return ASCHED_E_INVALID;
    const int ty = inst->veh_type ? inst->veh_type[v] : 0;
    if (ty < 0 || ty >= nt) return ASCHED_E_INVALID;
  }
  for (int m = 0; m < M; ++m) {
    const int pk = inst->pickup[m], d = inst->delivery[m];
    if (pk < 0 || pk >= L || d < 0 || d >= L || pk == d) return ASCHED_E_INVALID;
    if (inst->heli_only && (inst->heli_only[m] < 0 || inst->heli_only[m] > 1)) return ASCHED_E_INVALID;
  }
  const double lam = p->cap_mode == ASCHED_PENALTY ? static_cast<double>(p->lambda) : 0.0;
  const double bound = 2.0 * (2.0 * M + V + 2.0) * static_cast<double>(maxT) * (1.0 + lam);
  if (!(bound < 2147483648.0)) return ASCHED_E_OVERFLOW_GUARD;
  return ASCHED_OK;
}

int asched_plan(const asched_instance* inst, const asched_params* params, asched_plan_t* out) {
  if (!out) return ASCHED_E_INVALID;
  return make_plan(inst, params, false, true, out, nullptr);
}

namespace {
KParams solve_params(const int32_t* init_route_off, const int32_t* init_route, const asched_result* out) {
  KParams kp = {};
  kp.init_off = init_route_off;
  kp.init_route = init_route;
  kp.out_off = out->route_off;
  kp.out_route = out->route;
  kp.out_flight = out->flight;
  kp.out_over = out->overflow;
  kp.info = out->info;
  kp.traj_move = out->traj_move;
  kp.traj_z = out->traj_z;
  return kp;
}
}  // namespace

int asched_solve(const asched_instance* inst, const asched_params* params, const int32_t* init_route_off,
                 const int32_t* init_route, const asched_result* out, void* stream) {
  const asched_nvtx::Range nvtx_range("asched_solve");
  if (!out || !out->route_off || !out->route || !out->info) return ASCHED_E_INVALID;
  if ((init_route_off == nullptr) != (init_route == nullptr)) return ASCHED_E_INVALID;
  return launch(inst, params, false, solve_params(init_route_off, init_route, out), nullptr, 0, false, stream);
}

int asched_validate(const asched_instance* inst, const asched_params* params) {
  return asched_check_instance_host(inst, params);
}

int asched_workspace_bytes(const asched_instance* inst, const asched_params* params, size_t* bytes) {
  if (!bytes) return ASCHED_E_INVALID;
  asched_plan_t plan;
  const int rc = make_plan(inst, params, false, true, &plan, nullptr);
  if (rc != ASCHED_OK) return rc;
  *bytes = static_cast<size_t>(plan.workspace_bytes);
  return ASCHED_OK;
}

int asched_greedy_init(const asched_instance* inst, const asched_params* params, int32_t* route_off,
                       int32_t* route, int32_t* info, void* stream) {
  const asched_nvtx::Range nvtx_range("asched_greedy_init");
  if (!params || !route_off || !route || !info) return ASCHED_E_INVALID;
  asched_params p0 = *params;
  p0.iterations = 0;
  p0.grid_clusters = 1;
  asched_result out = {};
  out.route_off = route_off;
  out.route = route;
  out.info = info;
  return asched_solve(inst, &p0, nullptr, nullptr, &out, stream);
}

int asched_tabu_solve(const asched_instance* inst, const asched_params* params, const int32_t* init_route_off,
                      const int32_t* init_route, const asched_result* out, void* workspace, size_t workspace_bytes,
                      void* stream) {
  const asched_nvtx::Range nvtx_range("asched_tabu_solve");
  if (!out || !out->route_off || !out->route || !out->info) return ASCHED_E_INVALID;
  if ((init_route_off == nullptr) != (init_route == nullptr)) return ASCHED_E_INVALID;
  return launch(inst, params, false, solve_params(init_route_off, init_route, out), workspace, workspace_bytes, true,
                stream);
}

int asched_batch_workspace_bytes(int32_t n_instances, size_t* out) {
  if (!out || n_instances < 0) return ASCHED_E_INVALID;
  *out = sizeof(int32_t) * (static_cast<size_t>(n_instances) + 1);
  return ASCHED_OK;
}

int asched_solve_batch(const asched_batch* batch, const asched_params* params, const asched_batch_result* out,
                       void* workspace, size_t workspace_bytes, void* stream) {
  const asched_nvtx::Range nvtx_range("asched_solve_batch");
  return launch_batch(batch, params, out, workspace, workspace_bytes, stream);
}

int asched_solve_batch_static(const asched_batch* batch, const asched_params* params,
                              const asched_batch_result* out, void* stream) {
  const asched_nvtx::Range nvtx_range("asched_solve_batch_static");
  if (!batch) return ASCHED_E_INVALID;
  if (batch->n_instances > ASCHED_STATIC_BATCH_MAX) return ASCHED_E_TOO_LARGE;
  void* scratch = nullptr;
  const int rc = static_scratch(&scratch);
  if (rc != ASCHED_OK) return rc;
  return launch_batch(batch, params, out, scratch, sizeof(g_batch_scratch), stream);
}

int asched_server_sizes(int32_t max_loc, int32_t max_vehicles, int32_t max_missions, int32_t n_types,
                        int32_t* slot_words, int32_t* out_words) {
  if (!slot_words || !out_words || max_loc < 1 || max_vehicles < 1 || max_missions < 0 || n_types < 1 ||
      n_types > 2)
    return ASCHED_E_INVALID;
  *slot_words = serve_slot_words(max_loc, max_vehicles, max_missions, n_types);
  *out_words = serve_out_words(max_vehicles, max_missions);
  return ASCHED_OK;
}

int asched_serve(const asched_server* server, const asched_params* params, int64_t idle_timeout_ns,
                 int32_t max_ctas, void* stream) {
  const asched_nvtx::Range nvtx_range("asched_serve");
  return launch_serve(server, params, idle_timeout_ns, max_ctas, stream);
}

int asched_eval_neighbourhood(const asched_instance* inst, const asched_params* params,
                              const int32_t* route_off, const int32_t* route, const int32_t* tabu_until,
                              int32_t it, int32_t z_best, int32_t* delta_out, uint8_t* flags_out,
                              uint32_t* id_out, unsigned long long* best_key_out, int32_t* info,
                              void* stream) {
  const asched_nvtx::Range nvtx_range("asched_eval_neighbourhood");
  if (!route_off || !route || !delta_out || !flags_out || !best_key_out || !info) return ASCHED_E_INVALID;
  KParams kp = {};
  kp.init_off = route_off;
  kp.init_route = route;
  kp.tabu_in = tabu_until;
  kp.dbg_it = it;
  kp.dbg_zbest = z_best;
  kp.dbg_delta = delta_out;
  kp.dbg_flags = flags_out;
  kp.dbg_id = id_out;
  kp.dbg_key = best_key_out;
  kp.info = info;
  return launch(inst, params, true, kp, nullptr, 0, false, stream);
}

}  // extern "C"
