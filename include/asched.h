/*
 * asched.h - C ABI of the GB300 (sm_103a) Tabu search for air-ambulance fleet
 * scheduling (Tassone & Choudhury, "Algorithms for Optimizing Fleet Scheduling of
 * Air Ambulances", arXiv 2002.11710).
 *
 * The problem (Section 3): vehicles sit on bases; a mission is a pickup -> delivery
 * pair; each vehicle flies a closed route base -> p1 -> d1 -> ... -> pn -> dn -> base;
 * every mission is flown exactly once; the objective is the total flight time (obj_s)
 * under a per-vehicle duty cap (con6), optional arrive-by times (con7/con8) and
 * helicopter-only missions (con9). The method improved here is the Tabu search of
 * Algorithm 3 (Section 4.3), started from the greedy schedule of Algorithm 1
 * (Section 4.1), widened to the whole neighbourhood each iteration:
 *   R(m, y)   take mission m out of its route and put it immediately before node y;
 *             a node is a mission (id 0..M-1) or the end of vehicle v's route (M+v);
 *             y != m and y != the node after m.  Move id (m << 13) | y.
 *   S(m1,m2)  m1 < m2 exchange places (also within one route).
 *             Move id 0x80000000 | (m1 << 13) | m2.
 * There are M(M+V-2) + M(M-1)/2 moves. Each iteration applies the admissible move
 * with the least (delta, move id); admissible = feasible and (not tabu, or its
 * objective is strictly below the best so far). Applying a move at iteration it
 * makes (x, vehicle x left) tabu up to iteration it + tenure for every moved
 * mission x; a move is tabu when it puts a mission x on a vehicle v with
 * tabu_until[x][v] >= it. No admissible move: the iteration applies nothing.
 *
 * Conventions for every call below:
 *   - "device" pointers are CUDA device memory owned by the caller (for example
 *     PyTorch tensors); the library never allocates or frees memory and never
 *     creates a stream or an event. Device buffers must stay valid until the work
 *     queued on `stream` has finished.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Calls that launch work return as soon as it is queued.
 *   - Every int32 array is dense and C-ordered. Travel times are integer minutes.
 *   - Return value: ASCHED_OK, or a negative ASCHED_E_* for errors found on the host
 *     before anything is queued (nothing is then written). Errors found on the
 *     device are written to info[ASCHED_INFO_STATUS], readable once the stream has
 *     been synchronised; the other outputs are then unspecified.
 *   - The calls are thread-compatible: no global mutable state besides the per-kernel
 *     attribute setup, which is idempotent.
 */
#ifndef ASCHED_H
#define ASCHED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ASCHED_ABI_VERSION 2

/* Status codes. */
#define ASCHED_OK 0
#define ASCHED_E_INVALID (-1)          /* argument or instance data out of range */
#define ASCHED_E_TOO_LARGE (-2)        /* instance does not fit the on-chip layout */
#define ASCHED_E_OVERFLOW_GUARD (-3)   /* int32 objective could overflow (see below) */
#define ASCHED_E_INFEASIBLE_INIT (-4)  /* no feasible initial schedule */
#define ASCHED_E_TIMEOUT (-5)          /* a bounded device wait gave up */
#define ASCHED_E_CUDA (-6)             /* a CUDA runtime call failed */

/* Cap modes (the duty cap p of con6). */
#define ASCHED_HARD 0     /* flight(v) <= duty_cap is a constraint */
#define ASCHED_PENALTY 1  /* Z = sum flight + lambda * sum max(0, flight - duty_cap) */

/* Per-move flags written by asched_eval_neighbourhood. */
#define ASCHED_FLAG_FEASIBLE 1u
#define ASCHED_FLAG_TABU 2u
#define ASCHED_FLAG_ASPIRATION 4u  /* Z + delta < z_best */
#define ASCHED_FLAG_ADMISSIBLE 8u

#define ASCHED_SWAP_BIT 0x80000000u
#define ASCHED_NULL_MOVE 0xFFFFFFFFu

/* Layout of the int32 info[ASCHED_INFO_LEN] output. */
#define ASCHED_INFO_STATUS 0   /* ASCHED_OK or a negative device-side status */
#define ASCHED_INFO_Z_BEST 1   /* objective of the best schedule */
#define ASCHED_INFO_BEST_IT 2  /* iteration that reached it (-1 = initial schedule) */
#define ASCHED_INFO_Z_INIT 3   /* objective of the initial schedule */
#define ASCHED_INFO_Z_FINAL 4  /* objective after the last iteration */
#define ASCHED_INFO_ITERS 5    /* iterations completed */
#define ASCHED_INFO_LEN 8

/* One problem instance (Section 3). Sizes are host values; arrays are device memory.
 *   travel    [n_types][n_loc][n_loc] minutes, every entry >= 0; type 0 = helicopter,
 *             type 1 = plane (the l index of d_ijl in Eq. e1); n_types is 1 or 2.
 *   veh_base  [n_vehicles] base location of each vehicle.
 *   veh_type  [n_vehicles] 0 or 1 (b_k), or NULL for all helicopters.
 *   pickup, delivery [n_missions] locations, pickup != delivery.
 *   heli_only [n_missions] 1 = only a type-0 vehicle may fly it (rho), or NULL.
 *   deadline  [n_missions] arrive-by minute at the delivery (w_n), or NULL for none.
 *             With deadlines a vehicle leaves a delivery exactly at its w_n; a link
 *             u -> m needs dep(u) + T[end u][p_m] + T[p_m][d_m] <= w_m (dep(base) = 0)
 *             and the return needs dep(u) + T[end u][base] <= horizon.
 *   duty_cap  p, flight minutes per vehicle; horizon: 1440 for a 24 h day. */
typedef struct {
  int32_t n_loc;
  int32_t n_types;
  int32_t n_vehicles;
  int32_t n_missions;
  const int32_t* travel;
  const int32_t* veh_base;
  const int32_t* veh_type;
  const int32_t* pickup;
  const int32_t* delivery;
  const int32_t* heli_only;
  const int32_t* deadline;
  int32_t duty_cap;
  int32_t horizon;
} asched_instance;

/* Search parameters.
 *   tenure, iterations  >= 0.
 *   cap_mode            ASCHED_HARD or ASCHED_PENALTY; lambda >= 0 (PENALTY weight).
 *   cluster_size        CTAs cooperating on one instance (a thread-block cluster):
 *                       0 = automatic, else 1, 2, 4, 8 or 16. Results do not depend
 *                       on it.
 *   block_threads       0 = automatic, else a multiple of 32 in [64, 512].
 *   timeout_ns          bound on every wait between CTAs; 0 = 1 s.
 *   flags               0, or a combination of ASCHED_COMPACT_LAYOUT,
 *                       ASCHED_TEST_WITHHOLD_KEY and ASCHED_PLAIN_LAUNCH.
 *   grid_clusters       clusters cooperating on one instance in asched_tabu_solve: 0 =
 *                       automatic, else 1..1024, every cluster resident at once (else
 *                       ASCHED_E_TOO_LARGE). Neighbourhoods of more than 4 chunks of 32
 *                       items per warp of one 16-CTA cluster (about 65,000 moves and up)
 *                       spread over every cluster the device holds. The clusters exchange
 *                       one 64-bit key per iteration through the caller's workspace
 *                       (asched_workspace_bytes). Calls without a workspace (asched_solve,
 *                       asched_greedy_init, asched_eval_neighbourhood) take 0 or 1.
 *                       Results do not depend on it.
 * Shared-memory layout: instances whose location x mission gather tables fit in one
 * CTA's shared memory use them; larger ones (or all, with ASCHED_COMPACT_LAYOUT) keep
 * the travel matrix itself as int16 instead, which needs every travel time <= 32,767
 * (else ASCHED_E_TOO_LARGE on the device) and iterations + tenure <= 32,767 (else
 * ASCHED_E_TOO_LARGE from the call). Results do not depend on the layout. */
#define ASCHED_COMPACT_LAYOUT 1u
/* Failure-path test hook for a single-instance search with several CTAs: in the first
 * iteration the last CTA of the cluster (one cluster) or the last cluster (several
 * clusters) does not publish its key, so every CTA's bounded wait runs out after
 * timeout_ns and the call reports ASCHED_E_TIMEOUT (nothing faults or hangs). No effect
 * with one CTA. */
#define ASCHED_TEST_WITHHOLD_KEY 2u
/* Launch the clusters of a multi-cluster search (grid_clusters > 1) without the
 * cooperative attribute, for tools that cannot replay a cooperative cluster launch (a
 * profiler). Co-residency of the clusters is then not guaranteed: on a device busy with
 * other work, a cluster that cannot start in time makes the others' bounded waits run
 * out (ASCHED_E_TIMEOUT). Results are unchanged. */
#define ASCHED_PLAIN_LAUNCH 4u
typedef struct {
  int32_t tenure;
  int32_t iterations;
  int32_t cap_mode;
  int32_t lambda;
  int32_t cluster_size;
  int32_t block_threads;
  int64_t timeout_ns;
  uint32_t flags;
  int32_t grid_clusters;
} asched_params;

/* Launch shape the library would use for an instance (see asched_plan). */
typedef struct {
  int32_t cluster_size;
  int32_t block_threads;
  int32_t smem_bytes;  /* dynamic shared memory per CTA */
  int64_t moves_per_iteration;
  int32_t grid_clusters;   /* clusters of cluster_size CTAs (asched_tabu_solve) */
  int64_t workspace_bytes; /* device workspace asched_tabu_solve needs for this shape */
} asched_plan_t;

/* Outputs of asched_solve; all device memory.
 *   route_off [n_vehicles + 1], route [n_missions]: best schedule in CSR form; the
 *             missions of vehicle v in flying order are route[route_off[v] ..
 *             route_off[v+1]).
 *   flight, overflow [n_vehicles]: minutes flown and minutes over duty_cap, best
 *             schedule.
 *   info      [ASCHED_INFO_LEN] (layout above).
 *   traj_move [iterations] applied move id per iteration (ASCHED_NULL_MOVE when
 *             none), or NULL; traj_z [iterations] objective after it, or NULL. */
typedef struct {
  int32_t* route_off;
  int32_t* route;
  int32_t* flight;
  int32_t* overflow;
  int32_t* info;
  uint32_t* traj_move;
  int32_t* traj_z;
} asched_result;

/* ABI version of the loaded library (ASCHED_ABI_VERSION). Never fails. */
int asched_abi_version(void);

/* Static text for a status code (never NULL). */
const char* asched_status_string(int status);

/* Number of canonical moves M(M+V-2) + M(M-1)/2 (Section 4.3 widened as above).
 * Returns ASCHED_E_INVALID for negative sizes or NULL out. Host only. */
int asched_num_moves(int32_t n_missions, int32_t n_vehicles, int64_t* out);

/* Validate an instance whose arrays are HOST memory, with the checks the device
 * prologue makes: index ranges, pickup != delivery, travel >= 0, n_types in {1,2},
 * flags in {0,1}, and the int32 overflow guard
 *   2 (2M + V + 2) max(travel) (1 + lambda) < 2^31.
 * Returns ASCHED_OK or the status the device would report. Host only, no CUDA call. */
int asched_check_instance_host(const asched_instance* inst, const asched_params* params);

/* Launch shape and shared-memory footprint asched_tabu_solve takes for the given sizes
 * (array pointers are not read). Returns ASCHED_E_TOO_LARGE when the instance does not
 * fit on chip, ASCHED_E_CUDA if the device cannot be queried. */
int asched_plan(const asched_instance* inst, const asched_params* params, asched_plan_t* out);

/* Tabu search (Algorithm 3) on one instance, all iterations in one persistent
 * launch of one cluster of `cluster_size` CTAs on `stream` (asched_tabu_solve below
 * with no workspace: grid_clusters must be 0 or 1).
 *   init_route_off/init_route: device CSR initial schedule (must be feasible), or
 *             both NULL to start from the greedy schedule of Algorithm 1 (heli-only
 *             missions first, then by (deadline, id); each appended to the vehicle
 *             with the least objective increase that stays feasible, lowest index on
 *             ties).
 * Device-side status: ASCHED_E_INVALID (bad data), ASCHED_E_OVERFLOW_GUARD,
 * ASCHED_E_INFEASIBLE_INIT, ASCHED_E_TIMEOUT. */
int asched_solve(const asched_instance* inst, const asched_params* params,
                 const int32_t* init_route_off, const int32_t* init_route,
                 const asched_result* out, void* stream);

/* The same calls under the names of the problem statement's interface: host-side
 * validation, the device workspace of a search, Algorithm 1 alone, and the Tabu search.
 *   asched_validate        = asched_check_instance_host (HOST arrays, no CUDA call).
 *   asched_workspace_bytes bytes of device workspace asched_tabu_solve needs with these
 *                          sizes and params (the plan's workspace_bytes): 0 when the
 *                          search runs on one cluster (every piece of its state lives
 *                          in shared memory), else the slots of the keys the clusters
 *                          exchange each iteration (two buffers of 128-byte lines).
 *   asched_greedy_init     Algorithm 1 (Section 4.1) on the device: the greedy schedule
 *                          written as device CSR route_off [V + 1] / route [M] and its
 *                          objective etc. in info [ASCHED_INFO_LEN] (a search of 0
 *                          iterations); device status ASCHED_E_INFEASIBLE_INIT when a
 *                          mission fits no vehicle.
 *   asched_tabu_solve      the Tabu search on the launch shape of asched_plan, which may
 *                          span several clusters (grid_clusters). workspace: device
 *                          memory of at least asched_workspace_bytes, 128-byte aligned
 *                          (NULL and 0 when that is 0); the call zeroes it on `stream`
 *                          before the launch, and two searches in flight at once need
 *                          two workspaces. The launch is cooperative (unless
 *                          ASCHED_PLAIN_LAUNCH), so every cluster is resident at once; it
 *                          fails with ASCHED_E_CUDA otherwise. A kernel launched with
 *                          another shape than planned writes ASCHED_E_INVALID and returns.
 *                          Results equal asched_solve's bit for bit. */
int asched_validate(const asched_instance* inst, const asched_params* params);
int asched_workspace_bytes(const asched_instance* inst, const asched_params* params, size_t* bytes);
int asched_greedy_init(const asched_instance* inst, const asched_params* params, int32_t* route_off,
                       int32_t* route, int32_t* info, void* stream);
int asched_tabu_solve(const asched_instance* inst, const asched_params* params,
                      const int32_t* init_route_off, const int32_t* init_route,
                      const asched_result* out, void* workspace, size_t workspace_bytes,
                      void* stream);

/* Every canonical move of one schedule, for checking (one launch, no move applied).
 *   route_off/route  device CSR schedule (must be feasible).
 *   tabu_until       device [n_missions][n_vehicles] int32, or NULL for none tabu.
 *   it, z_best       iteration number and best objective for the tabu / aspiration
 *                    tests.
 *   delta_out        device [moves] int32: objective change of each move.
 *   flags_out        device [moves] uint8: ASCHED_FLAG_* bits.
 *   id_out           device [moves] uint32 move ids, or NULL.
 *   best_key_out     device [1] uint64: ((delta ^ 0x80000000) << 32) | id of the
 *                    move the search would apply, or all ones when none.
 *   info             device [ASCHED_INFO_LEN].
 * Moves are written in canonical order: R(m, y) by (m, y), then S(m1, m2) by
 * (m1, m2), which is increasing move id. */
int asched_eval_neighbourhood(const asched_instance* inst, const asched_params* params,
                              const int32_t* route_off, const int32_t* route,
                              const int32_t* tabu_until, int32_t it, int32_t z_best,
                              int32_t* delta_out, uint8_t* flags_out, uint32_t* id_out,
                              unsigned long long* best_key_out, int32_t* info, void* stream);

/* ---------------------------------------------------------------- batches ----------
 * Many independent instances solved by one persistent launch (instances taken largest
 * first from a device work queue; each solved by one CTA, or with cluster_size C in
 * {2, 4, 8, 16} by a thread-block cluster of C CTAs, as many clusters as the device
 * holds at once; results do not depend on C). The arrays of
 * all instances are concatenated; instance b owns
 *   locations  [loc_off[b], loc_off[b+1]),  L_b = loc_off[b+1] - loc_off[b]
 *   vehicles   [veh_off[b], veh_off[b+1]),  V_b >= 1
 *   missions   [mis_off[b], mis_off[b+1]),  M_b >= 0
 *   travel     n_types * L_b * L_b minutes starting at travel_off[b]
 * Location indices (veh_base, pickup, delivery) are local to the instance. The three
 * offset arrays are given twice: h_* in host memory (read by the call to size the
 * launch) and as device copies (read by the kernel); they must agree.
 * Every instance shares the asched_params (cluster_size 0 means 1 here). */
typedef struct {
  int32_t n_instances;
  int32_t n_types;
  const int32_t* h_loc_off;  /* HOST [n_instances + 1] */
  const int32_t* h_veh_off;  /* HOST [n_instances + 1] */
  const int32_t* h_mis_off;  /* HOST [n_instances + 1] */
  const int32_t* loc_off;    /* device [n_instances + 1] */
  const int32_t* veh_off;    /* device [n_instances + 1] */
  const int32_t* mis_off;    /* device [n_instances + 1] */
  const int64_t* travel_off; /* device [n_instances] */
  const int32_t* travel;     /* device, concatenated */
  const int32_t* veh_base;   /* device [veh_off[B]] */
  const int32_t* veh_type;   /* device [veh_off[B]] or NULL */
  const int32_t* pickup;     /* device [mis_off[B]] */
  const int32_t* delivery;   /* device [mis_off[B]] */
  const int32_t* heli_only;  /* device [mis_off[B]] or NULL */
  const int32_t* deadline;   /* device [mis_off[B]] or NULL (then no instance has deadlines) */
  const int32_t* duty_cap;   /* device [n_instances] */
  const int32_t* horizon;    /* device [n_instances] */
} asched_batch;

/* Outputs of asched_solve_batch (device memory), per instance b:
 *   route_off  V_b + 1 entries at route_off[veh_off[b] + b], offsets local to b
 *   route      M_b entries at route[mis_off[b]]
 *   flight, overflow  V_b entries at [veh_off[b]] (may be NULL)
 *   info       ASCHED_INFO_LEN entries at info[b * ASCHED_INFO_LEN] */
typedef struct {
  int32_t* route_off;
  int32_t* route;
  int32_t* flight;
  int32_t* overflow;
  int32_t* info;
} asched_batch_result;

/* Device workspace asched_solve_batch needs for n_instances (a queue counter and the
 * processing order): 4 * (n_instances + 1) bytes. Host only. */
int asched_batch_workspace_bytes(int32_t n_instances, size_t* out);

/* Tabu search (Algorithm 3, greedy start of Algorithm 1) on every instance of the
 * batch: one small ordering kernel, then one persistent launch on `stream`. Each
 * instance's result equals what asched_solve returns for it alone. workspace is
 * caller-owned device memory of at least asched_batch_workspace_bytes; it is
 * overwritten, and two batches in flight at once need two workspaces. Returns
 * ASCHED_E_TOO_LARGE if some instance does not fit the on-chip layout. */
int asched_solve_batch(const asched_batch* batch, const asched_params* params,
                       const asched_batch_result* out, void* workspace, size_t workspace_bytes,
                       void* stream);

/* ---------------------------------------------------------------- serving ----------
 * A persistent launch that solves requests while the host keeps admitting new ones
 * (continuous batching: every CTA takes the next published request as soon as it is
 * free, so requests that arrive while others run overlap with them on the device).
 *
 * Device memory, all caller-owned:
 *   slot_data [n_slots][slot_words]  request inputs; slot layout (int32 words):
 *       [0] n_loc  [1] n_vehicles  [2] n_missions  [3] duty_cap  [4] horizon
 *       [5] flags (1: heli_only present, 2: deadline present)  [6] sequence number
 *       [ASCHED_SLOT_HEADER ...] travel [n_types][n_loc][n_loc] (row length n_loc),
 *       then at ASCHED_SLOT_HEADER + n_types*max_loc^2: veh_base [max_vehicles],
 *       veh_type [max_vehicles], pickup [max_missions], delivery [max_missions],
 *       heli_only [max_missions], deadline [max_missions].
 *   slot_out [n_slots][out_words]  results: route_off [max_vehicles + 1], route
 *       [max_missions], flight [max_vehicles], overflow [max_vehicles], info
 *       [ASCHED_INFO_LEN].
 *   ring [ring_len]   slot index of ticket t at ring[t % ring_len] (ring_len >= n_slots).
 *   control [ASCHED_CTRL_LEN]  zeroed before the launch; the host raises
 *       control[ASCHED_CTRL_PUBLISHED] to publish tickets and sets
 *       control[ASCHED_CTRL_STOP] to end the launch; the launch counts served requests
 *       in control[ASCHED_CTRL_SERVED].
 *   done [n_slots]    the launch writes slot s's sequence number there when s is solved.
 * Publish a slot by copies ordered on one stream: slot contents, then its ring entry,
 * then the new published count. A slot may be rewritten once its sequence number has
 * appeared in done[]. Requests of one launch share asched_params, and either all or none
 * carry deadlines (has_deadlines). */
#define ASCHED_SLOT_HEADER 16
#define ASCHED_CTRL_PUBLISHED 0
#define ASCHED_CTRL_CLAIMED 1
#define ASCHED_CTRL_STOP 2
#define ASCHED_CTRL_SERVED 3
#define ASCHED_CTRL_IDLE_EXITS 4
#define ASCHED_CTRL_STARTED 5 /* CTAs of the launch that have started */
#define ASCHED_CTRL_LEN 8

typedef struct {
  int32_t n_slots;
  int32_t ring_len;
  int32_t max_loc;
  int32_t max_vehicles;
  int32_t max_missions;
  int32_t n_types;
  int32_t has_deadlines;
  int32_t* slot_data;
  int32_t* slot_out;
  int32_t* ring;
  int32_t* control;
  int32_t* done;
} asched_server;

/* Words per input slot and per output slot for the given capacities. Host only. */
int asched_server_sizes(int32_t max_loc, int32_t max_vehicles, int32_t max_missions, int32_t n_types,
                        int32_t* slot_words, int32_t* out_words);

/* Start the serving launch on `stream` (returns at once). max_ctas > 0 caps the number
 * of CTAs (default: every SM). With params->cluster_size C in {2, 4, 8, 16} the launch
 * is made of clusters of C CTAs (max_ctas / C of them, as many as the device places) and
 * each request is solved by a whole cluster, as asched_solve with that cluster size:
 * for the largest requests of a mixed stream, served by a second launch with its own
 * ring and control words over the same slots. Every CTA adds 1 to
 * control[ASCHED_CTRL_STARTED] when it starts. The call loads every serving kernel
 * first, so that a second serving launch started while one runs does not wait for it
 * (kernels load on first use, and a load can wait for the device to be idle). The launch
 * ends once control[ASCHED_CTRL_STOP] is set and every published request has been taken, or after idle_timeout_ns (> 0) without a new
 * request (counted in control[ASCHED_CTRL_IDLE_EXITS]). A request whose sizes exceed the
 * capacities, or whose deadline flag differs from has_deadlines, gets ASCHED_E_INVALID
 * in its info[ASCHED_INFO_STATUS]. */
int asched_serve(const asched_server* server, const asched_params* params, int64_t idle_timeout_ns,
                 int32_t max_ctas, void* stream);

/* Largest batch asched_solve_batch_static accepts. */
#define ASCHED_STATIC_BATCH_MAX 16384

/* asched_solve_batch without a caller workspace (no counterpart in the paper: it only
 * changes who provides scratch memory). For callers that cannot allocate device memory
 * themselves: a host program that embeds the solver with no device allocator of its
 * own, or a dispatch loop that must not call cudaMalloc because cudaMalloc can
 * synchronise the whole device and stall every other stream. The call allocates
 * nothing: its queue counter and processing order live in a fixed array of
 * 4 * (ASCHED_STATIC_BATCH_MAX + 1) bytes (64 KB) that every GPU using this library
 * holds until the process exits. The caller still provides every input and output.
 *   - Batches above ASCHED_STATIC_BATCH_MAX instances return ASCHED_E_TOO_LARGE.
 *   - Every call looks up the array's device address on the current device (a lookup,
 *     no allocation), so the address stays right after a device reset. The first call
 *     on a device may load the library's device code: make that first call before any
 *     stream capture on that device.
 *   - All calls on a device share the array and leave their contents in it (the next
 *     call resets what must start at zero), so two of these calls whose work overlaps
 *     on the GPU (different streams, not ordered) race with each other. Order them on
 *     one stream, or use asched_solve_batch with separate workspaces.
 * Results are those of asched_solve_batch. */
int asched_solve_batch_static(const asched_batch* batch, const asched_params* params,
                              const asched_batch_result* out, void* stream);

/* ---------------------------------------------------------------- sweeps -----------
 * The paper's own local searches in the per-mission sweep form it prints, on every
 * instance of a batch (one CTA per instance):
 *   ASCHED_SWEEP_NEIGHBOURHOOD  Algorithm 2 (Neighbourhood Search, Section 4.2);
 *   ASCHED_SWEEP_TABU           Algorithm 3 as printed (Section 4.3).
 * Each starts from the greedy schedule of Algorithm 1 and sweeps vehicles i = 0..V-1
 * in order; for i, the missions j of i's route as it stands when i's turn starts, in
 * route order (one step each, counted over the whole search), are relocated:
 *   - candidates: every other vehicle k whose type may fly j (con9), at every insertion
 *     point q = 0..n_k in order; the first q whose schedule breaks the duty cap (HARD)
 *     or an arrive-by time ends the scan of k (the listings' "continue to the next
 *     base" inside the position loop);
 *   - Algorithm 3 also skips every k with (j, k) on the tabu list; applying a move of
 *     j off vehicle i at step s puts (j, i) on the list through step s + tenure (no
 *     aspiration);
 *   - the least (delta, k, q) is applied when delta < 0; with ASCHED_SWEEP_ACCEPT_WORSE
 *     (Algorithm 3 only) it is applied whatever its delta.
 * Sweeps repeat while one applied a move (ACCEPT_WORSE: while one lowered the best
 * objective), at most params->iterations sweeps. The result is the first schedule
 * that reached the least objective. */
#define ASCHED_SWEEP_NEIGHBOURHOOD 2
#define ASCHED_SWEEP_TABU 3
#define ASCHED_SWEEP_ACCEPT_WORSE 4u /* asched_params.flags bit for the sweeps */
/* asched_params.flags bit for the sweeps: Algorithm 1's repair. When no vehicle can take
 * the next mission and some mission is already placed, one Neighbourhood Search sweep
 * (the rules above, on the partial schedule) runs and the mission is tried once more
 * (Section 4.1 leaves a stuck placement to "mission swaps" of Algorithm 2 and a retry).
 * Without it, or if the retry fails too, info[ASCHED_INFO_STATUS] is
 * ASCHED_E_INFEASIBLE_INIT. */
#define ASCHED_SWEEP_REPAIR 8u

/* info[] of a sweep: ASCHED_INFO_STATUS, _Z_BEST, _Z_INIT, _Z_FINAL as above;
 * ASCHED_INFO_BEST_IT = step that reached the best (-1: the greedy schedule);
 * ASCHED_INFO_ITERS = sweeps run; and: */
#define ASCHED_INFO_MOVES 6 /* moves applied */
#define ASCHED_INFO_STEPS 7 /* mission steps taken */

/* Optional per-step trace of a sweep (device memory): entry s of instance b at
 * [b * capacity + s] for s < capacity: the applied relocation id (j << 13) | y, y the
 * node j now precedes (a mission, or n_missions + k at the end of route k), or
 * ASCHED_NULL_MOVE; and the objective after the step. move or z may be NULL. */
typedef struct {
  uint32_t* move;
  int32_t* z;
  int32_t capacity;
} asched_sweep_trace;

/* Loop orders of the sweeps (device memory, optional). The paper lets the loops over
 * bases and over a base's missions run in random permutation order (Section 4.2); a run
 * of the sweeps takes one such pair of orders, kept for all its sweeps and for
 * Algorithm 1's repair sweep:
 *   vehicle_order  V_b entries at veh_off[b]: the vehicles' turns, a permutation of
 *                  0..V_b-1; NULL: 0, 1, ..., V_b-1.
 *   mission_rank   M_b entries at mis_off[b]: a vehicle's missions are tried by
 *                  increasing rank, a permutation of 0..M_b-1; NULL: route order.
 * An order that is not a permutation gives ASCHED_E_INVALID in that instance's status.
 * Several runs of one instance are several batch entries with different orders. */
typedef struct {
  const int32_t* vehicle_order;
  const int32_t* mission_rank;
} asched_sweep_orders;

/* Queue the sweep `algorithm` on every instance of `batch` on `stream`. params:
 * tenure (Algorithm 3), iterations = the most sweeps (>= 0), cap_mode, lambda,
 * cluster_size 0 or 1, block_threads 0 (automatic) or a multiple of 32 in [32, 512],
 * flags: ASCHED_SWEEP_ACCEPT_WORSE (Algorithm 3 only) and ASCHED_SWEEP_REPAIR; timeout_ns
 * is unused (the sweep waits on nothing). iterations * n_missions + tenure must stay below 2^31.
 * orders may be NULL (index and route order). out is laid out as for asched_solve_batch
 * (flight and overflow may be NULL); trace may be NULL. Instances whose state does not fit one CTA's shared memory return
 * ASCHED_E_TOO_LARGE (a paper-sized instance needs about 4 KB). */
int asched_sweep_batch(const asched_batch* batch, int32_t algorithm, const asched_params* params,
                       const asched_sweep_orders* orders, const asched_batch_result* out,
                       const asched_sweep_trace* trace, void* stream);

/* ---------------------------------------------------------------- travel matrix ----
 * Travel-time matrices built on the device from location coordinates (Eq. e1,
 * Section 3), written straight into the concatenated travel array of an asched_batch:
 *   travel[travel_off[b] + (t * L_b + i) * L_b + j] = rint(dist_km(i, j) / speed_kmh[t] * 60)
 * in float64, half to even, where L_b = loc_off[b + 1] - loc_off[b] and dist_km is
 *   ASCHED_METRIC_HAVERSINE  Eq. e1's great-circle distance, 2 r asin(sqrt(sin^2(dphi/2)
 *                            + cos(phi_i) cos(phi_j) sin^2(dpsi/2))), sqrt clipped to 1;
 *                            coords are (latitude, longitude) in degrees;
 *   ASCHED_METRIC_EUCLIDEAN  sqrt(dx^2 + dy^2) on (x, y) kilometres, every operation
 *                            rounded separately (identical to a float64 evaluation).
 * The Haversine path uses the device's sine, cosine and arcsine: a time within a few
 * ulps of a half minute may round the other way than on a host. */
#define ASCHED_METRIC_EUCLIDEAN 0
#define ASCHED_METRIC_HAVERSINE 1

typedef struct {
  int32_t n_instances;
  const int32_t* h_loc_off;  /* HOST [n_instances + 1], h_loc_off[0] = 0, every L_b >= 1 */
  const int32_t* loc_off;    /* device copy of h_loc_off */
  const int64_t* travel_off; /* device [n_instances]: start of instance b's block */
  const double* coords;      /* device [h_loc_off[B]][2] */
  int32_t n_types;           /* 1 or 2 */
  double speed_kmh[2];       /* per vehicle type, > 0 (the paper: 300 helicopter, 500 plane) */
  int32_t metric;            /* ASCHED_METRIC_* */
  double radius_km;          /* Haversine only; 0 = 6371 */
} asched_travel_spec;

/* Queue the matrices of every instance on `stream`. travel: device, laid out as
 * asched_batch.travel. status: device int32 or NULL; the call sets it to ASCHED_OK, and
 * the kernel to ASCHED_E_INVALID if a coordinate is not finite or a time does not fit
 * int32 (such entries are written as 0). */
int asched_travel_matrix(const asched_travel_spec* spec, int32_t* travel, int32_t* status, void* stream);

/* ---------------------------------------------------------------- roofline probes --
 * Microbenchmarks of one SM's integer issue rate and shared-memory load rate, the
 * denominators of the roofline of the search kernels (not part of the paper's method).
 * One launch fills every SM with resident CTAs of *threads_out threads; CTA c writes
 * rec[3c] = its SM id, rec[3c+1] and rec[3c+2] = that SM's clock (clock64) after a block
 * barrier before and after its work. Per thread the work is iters steps of
 *   ASCHED_PROBE_INT32       ASCHED_PROBE_INT32_OPS_PER_STEP int32 add / xor / min
 *                            operations (8 independent chains);
 *   ASCHED_PROBE_INT32_ADD_XOR  ASCHED_PROBE_INT32_ADD_XOR_OPS_PER_STEP int32 add / xor
 *                            operations (8 independent chains; no min, which issues on
 *                            fewer pipes);
 *   ASCHED_PROBE_LDS         ASCHED_PROBE_LDS_LOADS_PER_STEP 32-bit shared-memory loads,
 *                            the 32 lanes of a warp on 32 distinct banks;
 *   ASCHED_PROBE_LDS_GATHER  as many loads, each lane at a random word of a 64 KB table.
 * A rate per SM is (CTAs on the SM) * threads * iters * (work per step) / (last end -
 * first start on that SM). rec: device int64 [3 * rec_ctas]; sink: device uint32
 * [rec_ctas] (written only in practice-impossible cases, to keep the work live);
 * *ctas_out = CTAs launched (ASCHED_E_INVALID if above rec_ctas). Asynchronous on
 * `stream`. */
#define ASCHED_PROBE_INT32 0
#define ASCHED_PROBE_LDS 1
#define ASCHED_PROBE_LDS_GATHER 2
#define ASCHED_PROBE_INT32_ADD_XOR 3
#define ASCHED_PROBE_INT32_OPS_PER_STEP 96
#define ASCHED_PROBE_INT32_ADD_XOR_OPS_PER_STEP 64
#define ASCHED_PROBE_LDS_LOADS_PER_STEP 16
int asched_probe_sm_peak(int32_t kind, int32_t iters, int64_t* rec, int32_t rec_ctas, uint32_t* sink,
                         int32_t* ctas_out, int32_t* threads_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ASCHED_H */
