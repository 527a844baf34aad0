/*
 * Plain CPU oracle for the Tabu search of Tassone & Choudhury, "Algorithms for
 * Optimizing Fleet Scheduling of Air Ambulances" (arXiv 2002.11710).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library. The product path
 * never calls it and shares no code with it.
 *
 * Everything here is written the slow, obvious way:
 *   - a schedule is one ordered mission list per vehicle;
 *   - a move is applied by building the new schedule explicitly;
 *   - the objective of every candidate schedule is recomputed from scratch as
 *     the sum of its legs (objective obj_s, Section 3), in 64-bit integers;
 *   - feasibility of every candidate is checked over the whole schedule
 *     (constraints con1-con9, Section 3, with the readings listed below).
 * Nothing uses an incremental delta formula.
 *
 * Readings of the paper taken here (the paper is silent or garbled on these):
 *   R1  A route of vehicle v is base(v) -> p1 -> d1 -> ... -> pn -> dn -> base(v);
 *       an empty route flies 0 minutes. Leg times come from the travel layer of
 *       the vehicle's type (l = b_k in obj_s).
 *   R2  Cap mode HARD: flight(v) <= p for every v (con6). Cap mode PENALTY:
 *       Z = sum flight + lambda * sum max(0, flight - p); the cap is then no
 *       constraint. Compatibility and deadlines are constraints in both modes.
 *   R3  Compatibility (con9): a heli-only mission never flies on a type-1 (plane)
 *       vehicle.
 *   R4  Deadlines (con7/con8, Section 3 text): w_m is the arrive-by time at the
 *       delivery of m; the vehicle leaves m's delivery exactly at w_m. A link
 *       u -> m is feasible iff dep(u) + T[end u][p_m] + T[p_m][d_m] <= w_m with
 *       dep(base) = 0, dep(m') = w_m'. The return link needs dep(u) + T[end u][base]
 *       <= horizon (24 h). con8's product is read as a sum.
 *   R5  The neighbourhood (Algorithm 3 widened to the whole neighbourhood):
 *         R(m, y): take mission m out of its route and put it immediately before
 *                  node y, where a node is a mission (id 0..M-1) or the end of the
 *                  route of vehicle v (id M+v); y != m and y != the node after m.
 *         S(m1, m2), m1 < m2: the two missions exchange places.
 *       Move ids: R = (m << 13) | y,  S = 2^31 | (m1 << 13) | m2 (unsigned).
 *   R6  Tabu attribute (TabuList/TabuCounter, Algorithm 3): the pair (mission,
 *       vehicle the mission left). Applying a move at iteration it sets
 *       tabu_until[x][from(x)] = it + tenure for every moved mission x. A move is
 *       tabu at iteration it iff some mission x it places on vehicle v has
 *       tabu_until[x][v] >= it. Aspiration: a tabu move is still admissible when
 *       its objective is strictly below the best found so far.
 *   R7  Each iteration applies the admissible move with the least (delta, move
 *       id); when no move is admissible the iteration applies nothing. The best
 *       schedule is replaced only on a strict improvement (earliest kept).
 *   R8  Initial schedule (Algorithm 1): heli-only missions first, then the rest,
 *       each group by (deadline, mission id) (by id when there are no deadlines);
 *       each mission is appended to the end of the route of the vehicle with the
 *       least increase of the objective among the vehicles that stay feasible,
 *       ties to the lowest vehicle index. No feasible vehicle is an error (the
 *       paper's swap repair is not taken).
 *   R12 Algorithm 1's repair, an option used by the sweeps (Section 4.1 leaves it to
 *       "mission swaps" of Algorithm 2 and a retry): when no vehicle can take mission m
 *       and some mission is already placed, one sweep of Algorithm 2 (readings S1-S3)
 *       runs over the partial schedule, and m is tried once more if the sweep moved
 *       anything. No vehicle after that, or no mission placed yet, is the error.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_E_INVALID (-1)
#define ORC_E_INFEASIBLE_INIT (-4)
#define ORC_E_NOMEM (-9)

#define ORC_HARD 0
#define ORC_PENALTY 1

#define ORC_FEASIBLE 1u
#define ORC_TABU 2u
#define ORC_ASPIRATION 4u
#define ORC_ADMISSIBLE 8u

#define ORC_SWAP_BIT 0x80000000u
#define ORC_NULL_MOVE 0xFFFFFFFFu

typedef struct {
  int32_t n_loc, n_types, n_vehicles, n_missions;
  const int32_t *travel;    /* [n_types][n_loc][n_loc] */
  const int32_t *veh_base;  /* [V] */
  const int32_t *veh_type;  /* [V] */
  const int32_t *pickup;    /* [M] */
  const int32_t *delivery;  /* [M] */
  const int32_t *heli_only; /* [M] or NULL */
  const int32_t *deadline;  /* [M] or NULL */
  int32_t duty_cap, horizon, cap_mode, lambda;
} orc_instance;

/* One ordered mission list per vehicle: seq[v*M + k] is the k-th mission of v. */
typedef struct {
  int32_t V, M;
  int32_t *len;
  int32_t *seq;
} sched;

static int32_t tt(const orc_instance *in, int type, int i, int j) {
  return in->travel[((int64_t)type * in->n_loc + i) * in->n_loc + j];
}

static int sched_alloc(sched *s, int V, int M) {
  s->V = V;
  s->M = M;
  s->len = (int32_t *)calloc((size_t)V, sizeof(int32_t));
  s->seq = (int32_t *)calloc((size_t)V * (size_t)(M > 0 ? M : 1), sizeof(int32_t));
  return (s->len && s->seq) ? ORC_OK : ORC_E_NOMEM;
}

static void sched_free(sched *s) {
  free(s->len);
  free(s->seq);
  s->len = s->seq = NULL;
}

static void sched_copy(sched *dst, const sched *src) {
  memcpy(dst->len, src->len, sizeof(int32_t) * (size_t)src->V);
  for (int v = 0; v < src->V; v++)
    memcpy(dst->seq + (int64_t)v * src->M, src->seq + (int64_t)v * src->M,
           sizeof(int32_t) * (size_t)src->len[v]);
}

static int sched_from_csr(sched *s, const int32_t *off, const int32_t *route) {
  if (off[0] != 0 || off[s->V] != s->M) return ORC_E_INVALID;
  for (int v = 0; v < s->V; v++) {
    int n = off[v + 1] - off[v];
    if (n < 0) return ORC_E_INVALID;
    s->len[v] = n;
    for (int k = 0; k < n; k++) s->seq[v * s->M + k] = route[off[v] + k];
  }
  return ORC_OK;
}

static void sched_to_csr(const sched *s, int32_t *off, int32_t *route) {
  off[0] = 0;
  for (int v = 0; v < s->V; v++) {
    for (int k = 0; k < s->len[v]; k++) route[off[v] + k] = s->seq[v * s->M + k];
    off[v + 1] = off[v] + s->len[v];
  }
}

/* Where mission m sits: vehicle and index. Returns 0 if it is not found. */
static int locate(const sched *s, int m, int *v_out, int *k_out) {
  for (int v = 0; v < s->V; v++)
    for (int k = 0; k < s->len[v]; k++)
      if (s->seq[v * s->M + k] == m) {
        *v_out = v;
        *k_out = k;
        return 1;
      }
  return 0;
}

/* Flight minutes of vehicle v flying `n` missions `ms` in order (R1, obj_s). */
static int64_t route_flight(const orc_instance *in, int v, const int32_t *ms, int n) {
  if (n == 0) return 0;
  int ty = in->veh_type[v], b = in->veh_base[v];
  int64_t f = tt(in, ty, b, in->pickup[ms[0]]);
  for (int k = 0; k < n; k++) {
    int m = ms[k];
    f += tt(in, ty, in->pickup[m], in->delivery[m]);
    if (k + 1 < n) f += tt(in, ty, in->delivery[m], in->pickup[ms[k + 1]]);
  }
  f += tt(in, ty, in->delivery[ms[n - 1]], b);
  return f;
}

static int64_t over_cap(const orc_instance *in, int64_t flight) {
  int64_t o = flight - in->duty_cap;
  return o > 0 ? o : 0;
}

/* Objective Z of a whole schedule (obj_s plus the PENALTY reading R2). */
static int64_t sched_cost(const orc_instance *in, const sched *s, int64_t *flight_out,
                          int64_t *over_out) {
  int64_t z = 0, pen = 0;
  for (int v = 0; v < s->V; v++) {
    int64_t f = route_flight(in, v, s->seq + (int64_t)v * s->M, s->len[v]);
    int64_t o = over_cap(in, f);
    if (flight_out) flight_out[v] = f;
    if (over_out) over_out[v] = o;
    z += f;
    pen += o;
  }
  if (in->cap_mode == ORC_PENALTY) z += (int64_t)in->lambda * pen;
  return z;
}

/* Deadline feasibility of one route (R4). */
static int route_deadlines_ok(const orc_instance *in, int v, const int32_t *ms, int n) {
  if (!in->deadline || n == 0) return 1;
  int ty = in->veh_type[v], b = in->veh_base[v];
  int64_t dep = 0;
  int end = b;
  for (int k = 0; k < n; k++) {
    int m = ms[k];
    int64_t arrive = dep + tt(in, ty, end, in->pickup[m]) + tt(in, ty, in->pickup[m], in->delivery[m]);
    if (arrive > in->deadline[m]) return 0;
    dep = in->deadline[m];
    end = in->delivery[m];
  }
  return dep + tt(in, ty, end, b) <= in->horizon;
}

/* The per-route constraints alone: compatibility (con9, R3), deadlines (con7/con8,
 * R4) and in HARD mode the duty cap (con6). Also meaningful for a partial schedule
 * (Algorithm 1 while it still places missions). */
static int routes_feasible(const orc_instance *in, const sched *s) {
  for (int v = 0; v < s->V; v++) {
    const int32_t *ms = s->seq + (int64_t)v * s->M;
    for (int k = 0; k < s->len[v]; k++)
      if (in->heli_only && in->heli_only[ms[k]] && in->veh_type[v] != 0) return 0;
    if (!route_deadlines_ok(in, v, ms, s->len[v])) return 0;
    if (in->cap_mode == ORC_HARD && route_flight(in, v, ms, s->len[v]) > in->duty_cap) return 0;
  }
  return 1;
}

/* Whole-schedule feasibility: every mission exactly once (con1/con2), compatibility
 * (con9, R3), deadlines (con7/con8, R4), and in HARD mode the duty cap (con6). */
static int sched_feasible(const orc_instance *in, const sched *s) {
  int M = s->M;
  int *seen = (int *)calloc((size_t)(M > 0 ? M : 1), sizeof(int));
  if (!seen) return 0;
  int ok = 1;
  for (int v = 0; v < s->V && ok; v++) {
    const int32_t *ms = s->seq + (int64_t)v * M;
    for (int k = 0; k < s->len[v]; k++) {
      int m = ms[k];
      if (m < 0 || m >= M || seen[m]) { ok = 0; break; }
      seen[m] = 1;
      if (in->heli_only && in->heli_only[m] && in->veh_type[v] != 0) { ok = 0; break; }
    }
    if (!ok) break;
    if (!route_deadlines_ok(in, v, ms, s->len[v])) ok = 0;
    if (in->cap_mode == ORC_HARD && route_flight(in, v, ms, s->len[v]) > in->duty_cap) ok = 0;
  }
  for (int m = 0; m < M && ok; m++)
    if (!seen[m]) ok = 0;
  free(seen);
  return ok;
}

/* The node that follows mission m in its route: the next mission, or M+v at the end. */
static int succ_node(const sched *s, int m) {
  int v, k;
  if (!locate(s, m, &v, &k)) return -1;
  if (k + 1 < s->len[v]) return s->seq[v * s->M + k + 1];
  return s->M + v;
}

static void remove_at(sched *s, int v, int k) {
  int32_t *ms = s->seq + (int64_t)v * s->M;
  for (int j = k; j + 1 < s->len[v]; j++) ms[j] = ms[j + 1];
  s->len[v]--;
}

static void insert_at(sched *s, int v, int k, int m) {
  int32_t *ms = s->seq + (int64_t)v * s->M;
  for (int j = s->len[v]; j > k; j--) ms[j] = ms[j - 1];
  ms[k] = m;
  s->len[v]++;
}

typedef struct {
  int n;
  int mission[2], from[2], to[2];
} moved_t;

/* Build the schedule a move leads to (R5). Returns 0 for an id that is not a move
 * of this schedule. */
static int apply_move(const orc_instance *in, const sched *s, uint32_t id, sched *t, moved_t *mv) {
  int M = s->M, V = s->V;
  sched_copy(t, s);
  if (id & ORC_SWAP_BIT) {
    int m1 = (int)((id >> 13) & 0x3FFFFu), m2 = (int)(id & 0x1FFFu);
    int v1, k1, v2, k2;
    if (m1 >= m2 || m2 >= M) return 0;
    if (!locate(s, m1, &v1, &k1) || !locate(s, m2, &v2, &k2)) return 0;
    t->seq[v1 * M + k1] = m2;
    t->seq[v2 * M + k2] = m1;
    mv->n = 2;
    mv->mission[0] = m1; mv->from[0] = v1; mv->to[0] = v2;
    mv->mission[1] = m2; mv->from[1] = v2; mv->to[1] = v1;
    return 1;
  }
  int m = (int)(id >> 13), y = (int)(id & 0x1FFFu);
  int vm, km;
  if (m >= M || y >= M + V || y == m) return 0;
  if (!locate(s, m, &vm, &km)) return 0;
  if (y == succ_node(s, m)) return 0;
  remove_at(t, vm, km);
  int vt;
  if (y < M) {
    int ky;
    if (!locate(t, y, &vt, &ky)) return 0;
    insert_at(t, vt, ky, m);
  } else {
    vt = y - M;
    insert_at(t, vt, t->len[vt], m);
  }
  mv->n = 1;
  mv->mission[0] = m; mv->from[0] = vm; mv->to[0] = vt;
  (void)in;
  return 1;
}

/* The canonical move list of a schedule, in increasing id order (R5). */
static int64_t enumerate_moves(const sched *s, uint32_t *ids) {
  int M = s->M, V = s->V;
  int64_t n = 0;
  for (int m = 0; m < M; m++) {
    int nx = succ_node(s, m);
    for (int y = 0; y < M + V; y++) {
      if (y == m || y == nx) continue;
      if (ids) ids[n] = ((uint32_t)m << 13) | (uint32_t)y;
      n++;
    }
  }
  for (int m1 = 0; m1 < M; m1++)
    for (int m2 = m1 + 1; m2 < M; m2++) {
      if (ids) ids[n] = ORC_SWAP_BIT | ((uint32_t)m1 << 13) | (uint32_t)m2;
      n++;
    }
  return n;
}

static int check_instance(const orc_instance *in) {
  if (in->n_loc <= 0 || in->n_types < 1 || in->n_types > 2 || in->n_vehicles < 1 ||
      in->n_missions < 0 || in->n_missions > 8191 || in->n_missions + in->n_vehicles > 8192)
    return ORC_E_INVALID;
  for (int v = 0; v < in->n_vehicles; v++) {
    if (in->veh_base[v] < 0 || in->veh_base[v] >= in->n_loc) return ORC_E_INVALID;
    if (in->veh_type[v] < 0 || in->veh_type[v] >= in->n_types) return ORC_E_INVALID;
  }
  for (int m = 0; m < in->n_missions; m++) {
    if (in->pickup[m] < 0 || in->pickup[m] >= in->n_loc) return ORC_E_INVALID;
    if (in->delivery[m] < 0 || in->delivery[m] >= in->n_loc) return ORC_E_INVALID;
    if (in->pickup[m] == in->delivery[m]) return ORC_E_INVALID;
  }
  return ORC_OK;
}

/* ---------------------------------------------------------------- exported calls -- */

int64_t orc_num_moves(int32_t M, int32_t V) {
  sched s;
  if (sched_alloc(&s, V, M) != ORC_OK) return -1;
  /* Any schedule has the same count; put every mission on vehicle 0. */
  for (int m = 0; m < M; m++) s.seq[m] = m;
  s.len[0] = M;
  int64_t n = enumerate_moves(&s, NULL);
  sched_free(&s);
  return n;
}

/* Objective of a CSR schedule; per-vehicle flight and overflow out (may be NULL). */
int64_t orc_cost(const orc_instance *in, const int32_t *off, const int32_t *route,
                 int64_t *flight_out, int64_t *over_out) {
  sched s;
  if (sched_alloc(&s, in->n_vehicles, in->n_missions) != ORC_OK) return INT64_MIN;
  int64_t z = INT64_MIN;
  if (sched_from_csr(&s, off, route) == ORC_OK) z = sched_cost(in, &s, flight_out, over_out);
  sched_free(&s);
  return z;
}

int32_t orc_feasible(const orc_instance *in, const int32_t *off, const int32_t *route) {
  sched s;
  if (sched_alloc(&s, in->n_vehicles, in->n_missions) != ORC_OK) return 0;
  int ok = sched_from_csr(&s, off, route) == ORC_OK && sched_feasible(in, &s);
  sched_free(&s);
  return ok;
}

/* Algorithm 1 under reading R8. */
/* State of the per-mission sweeps (Algorithms 2 and 3, readings S1-S5 below). */
typedef struct {
  int use_tabu, accept_worse;
  int32_t tenure;
  int64_t *tabu; /* [M][V]: step through which (mission, vehicle) is tabu, or NULL */
  int64_t step, n_moves, best_step, z, z_best;
  sched *best; /* copy of the best schedule met, or NULL */
  uint32_t *trace_move;
  int64_t *trace_z;
  int64_t trace_cap;
  const int32_t *vorder; /* [V] order of the vehicles' turns, or NULL for 0..V-1 (S1) */
  const int32_t *mrank;  /* [M] rank of each mission within its vehicle's turn, or NULL (S1) */
} sweep_ctx;

/* One sweep over s (readings S1, S2 and S3 / S4 / S4b). s may be partial: missions that
 * Algorithm 1 has not placed yet are absent and play no part. Returns 1 when a move was
 * applied. */
static int sweep_pass(const orc_instance *in, sched *s, sched *t, int32_t *snap, sweep_ctx *c) {
  int M = s->M, V = s->V, applied = 0;
  for (int ii = 0; ii < V; ii++) {
    int i = c->vorder ? c->vorder[ii] : ii;
    int ni = s->len[i];
    memcpy(snap, s->seq + (int64_t)i * M, sizeof(int32_t) * (size_t)ni);
    if (c->mrank) /* the turn's missions by increasing rank (plain insertion sort) */
      for (int x = 1; x < ni; x++)
        for (int y = x; y > 0 && c->mrank[snap[y]] < c->mrank[snap[y - 1]]; y--) {
          int tmp = snap[y];
          snap[y] = snap[y - 1];
          snap[y - 1] = tmp;
        }
    for (int jj = 0; jj < ni; jj++) {
      int j = snap[jj], vj, kj;
      uint32_t rec = ORC_NULL_MOVE;
      if (locate(s, j, &vj, &kj) && vj == i) {
        int best_k = -1, best_q = -1;
        int64_t best_d = 0;
        for (int k = 0; k < V; k++) {
          if (k == i) continue;
          if (in->heli_only && in->heli_only[j] && in->veh_type[k] != 0) continue;
          if (c->use_tabu && c->tabu[(int64_t)j * V + k] >= c->step) continue; /* S4 */
          for (int q = 0; q <= s->len[k]; q++) {
            sched_copy(t, s);
            remove_at(t, i, kj);
            insert_at(t, k, q, j);
            if (!routes_feasible(in, t)) break; /* S2 */
            int64_t d = sched_cost(in, t, NULL, NULL) - c->z;
            if (best_k < 0 || d < best_d) {
              best_k = k;
              best_q = q;
              best_d = d;
            }
          }
        }
        if (best_k >= 0 && (best_d < 0 || c->accept_worse)) {
          int y = best_q < s->len[best_k] ? s->seq[(int64_t)best_k * M + best_q] : M + best_k;
          remove_at(s, i, kj);
          insert_at(s, best_k, best_q, j);
          c->z = sched_cost(in, s, NULL, NULL);
          if (c->use_tabu) c->tabu[(int64_t)j * V + i] = c->step + c->tenure;
          rec = ((uint32_t)j << 13) | (uint32_t)y;
          c->n_moves++;
          applied = 1;
          if (c->z < c->z_best) {
            c->z_best = c->z;
            c->best_step = c->step;
            if (c->best) sched_copy(c->best, s);
          }
        }
      }
      if (c->step < c->trace_cap) {
        if (c->trace_move) c->trace_move[c->step] = rec;
        if (c->trace_z) c->trace_z[c->step] = c->z;
      }
      c->step++;
    }
  }
  return applied;
}

/* The vehicle Algorithm 1 appends mission m to: least objective increase among the
 * vehicles whose route stays feasible, ties to the lowest index; -1 when none. */
static int greedy_pick(const orc_instance *in, const sched *s, sched *t, int m) {
  int best_v = -1;
  int64_t best_score = 0;
  int64_t z_before = sched_cost(in, s, NULL, NULL);
  for (int v = 0; v < s->V; v++) {
    sched_copy(t, s);
    insert_at(t, v, t->len[v], m);
    const int32_t *ms = t->seq + (int64_t)v * s->M;
    if (in->heli_only && in->heli_only[m] && in->veh_type[v] != 0) continue;
    if (!route_deadlines_ok(in, v, ms, t->len[v])) continue;
    if (in->cap_mode == ORC_HARD && route_flight(in, v, ms, t->len[v]) > in->duty_cap) continue;
    int64_t score = sched_cost(in, t, NULL, NULL) - z_before;
    if (best_v < 0 || score < best_score) {
      best_v = v;
      best_score = score;
    }
  }
  return best_v;
}

/* Algorithm 1 (reading R8, and R12 when `repair` is set, its sweep in the given orders). */
static int greedy_core(const orc_instance *in, int repair, const int32_t *vorder, const int32_t *mrank,
                       int32_t *off_out, int32_t *route_out) {
  int rc = check_instance(in);
  if (rc != ORC_OK) return rc;
  int M = in->n_missions, V = in->n_vehicles;
  sched s, t;
  if (sched_alloc(&s, V, M) != ORC_OK || sched_alloc(&t, V, M) != ORC_OK) return ORC_E_NOMEM;
  /* Mission order: heli-only first, then by deadline, then by id (plain selection sort). */
  int *order = (int *)malloc(sizeof(int) * (size_t)(M > 0 ? M : 1));
  int *used = (int *)calloc((size_t)(M > 0 ? M : 1), sizeof(int));
  int32_t *snap = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
  for (int k = 0; k < M; k++) {
    int best = -1;
    for (int m = 0; m < M; m++) {
      if (used[m]) continue;
      if (best < 0) { best = m; continue; }
      int hm = in->heli_only ? !in->heli_only[m] : 1, hb = in->heli_only ? !in->heli_only[best] : 1;
      int64_t wm = in->deadline ? in->deadline[m] : 0, wb = in->deadline ? in->deadline[best] : 0;
      if (hm < hb || (hm == hb && (wm < wb || (wm == wb && m < best)))) best = m;
    }
    used[best] = 1;
    order[k] = best;
  }
  rc = ORC_OK;
  for (int k = 0; k < M && rc == ORC_OK; k++) {
    int m = order[k];
    int v = greedy_pick(in, &s, &t, m);
    if (v < 0 && repair && k > 0) {
      /* R12: one sweep of Algorithm 2 over the partial schedule, then one more try. */
      sweep_ctx c = {0};
      c.best_step = -1;
      c.z = c.z_best = sched_cost(in, &s, NULL, NULL);
      c.vorder = vorder;
      c.mrank = mrank;
      if (sweep_pass(in, &s, &t, snap, &c)) v = greedy_pick(in, &s, &t, m);
    }
    if (v < 0) rc = ORC_E_INFEASIBLE_INIT;
    else insert_at(&s, v, s.len[v], m);
  }
  if (rc == ORC_OK) sched_to_csr(&s, off_out, route_out);
  free(order);
  free(used);
  free(snap);
  sched_free(&s);
  sched_free(&t);
  return rc;
}

/* Algorithm 1 as read in R8 (no repair). */
int32_t orc_greedy_init(const orc_instance *in, int32_t *off_out, int32_t *route_out) {
  return greedy_core(in, 0, NULL, NULL, off_out, route_out);
}

/* Algorithm 1 with the repair of R12. */
int32_t orc_greedy_init_repair(const orc_instance *in, int32_t *off_out, int32_t *route_out) {
  return greedy_core(in, 1, NULL, NULL, off_out, route_out);
}

/* Every canonical move of a schedule: delta = Z(after) - Z(before), flags (feasible,
 * tabu, aspiration, admissible) and id, in canonical order. Writes the index of the
 * chosen move (least (delta, id) among admissible moves, or -1) to *chosen_out.
 * Returns the number of moves, or a negative status.
 * The moves are evaluated independently of one another, each on its own copy of the
 * schedule, so the loop over them runs on OpenMP threads (orc_set_threads); the least
 * admissible move is then picked by one thread in canonical order, so the result does
 * not depend on the number of threads. */
int64_t orc_eval_neighbourhood(const orc_instance *in, const int32_t *off, const int32_t *route,
                               const int32_t *tabu_until, int32_t it, int64_t z_best,
                               int64_t *delta_out, uint8_t *flags_out, uint32_t *id_out,
                               int64_t *chosen_out) {
  int rc = check_instance(in);
  if (rc != ORC_OK) return rc;
  int M = in->n_missions, V = in->n_vehicles;
  sched s;
  if (sched_alloc(&s, V, M) != ORC_OK) return ORC_E_NOMEM;
  if (sched_from_csr(&s, off, route) != ORC_OK) {
    sched_free(&s);
    return ORC_E_INVALID;
  }
  int64_t n = enumerate_moves(&s, NULL);
  size_t nn = (size_t)(n > 0 ? n : 1);
  uint32_t *ids = (uint32_t *)malloc(sizeof(uint32_t) * nn);
  int64_t *delta = delta_out ? delta_out : (int64_t *)malloc(sizeof(int64_t) * nn);
  uint8_t *flags = flags_out ? flags_out : (uint8_t *)malloc(nn);
  if (!ids || !delta || !flags) rc = ORC_E_NOMEM;
  int64_t z0 = 0;
  if (rc == ORC_OK) {
    enumerate_moves(&s, ids);
    z0 = sched_cost(in, &s, NULL, NULL);
  }
  int bad = 0;  /* a thread without memory, or an id that is not a move */
#pragma omp parallel if (rc == ORC_OK && n > 1)
  {
    sched t;
    int ok = rc == ORC_OK && sched_alloc(&t, V, M) == ORC_OK;
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; i++) {
      moved_t mv;
      if (!ok || !apply_move(in, &s, ids[i], &t, &mv)) {
#pragma omp atomic write
        bad = 1;
        continue;
      }
      int64_t z1 = sched_cost(in, &t, NULL, NULL);
      unsigned fl = 0;
      if (sched_feasible(in, &t)) fl |= ORC_FEASIBLE;
      for (int j = 0; j < mv.n; j++)
        if (tabu_until[(int64_t)mv.mission[j] * V + mv.to[j]] >= it) fl |= ORC_TABU;
      if (z1 < z_best) fl |= ORC_ASPIRATION;
      if ((fl & ORC_FEASIBLE) && (!(fl & ORC_TABU) || (fl & ORC_ASPIRATION))) fl |= ORC_ADMISSIBLE;
      delta[i] = z1 - z0;
      flags[i] = (uint8_t)fl;
    }
    if (ok) sched_free(&t);
  }
  if (rc == ORC_OK && bad) rc = ORC_E_INVALID;
  int64_t chosen = -1;
  if (rc == ORC_OK) {
    for (int64_t i = 0; i < n; i++) {
      if (id_out) id_out[i] = ids[i];
      if ((flags[i] & ORC_ADMISSIBLE) &&
          (chosen < 0 || delta[i] < delta[chosen] || (delta[i] == delta[chosen] && ids[i] < ids[chosen])))
        chosen = i;
    }
  }
  if (chosen_out) *chosen_out = chosen;
  free(ids);
  if (!delta_out) free(delta);
  if (!flags_out) free(flags);
  sched_free(&s);
  return rc == ORC_OK ? n : rc;
}

/* Threads of the OpenMP loop over moves (n <= 0: one per processor); returns the
 * number now in force (1 when built without OpenMP). */
int32_t orc_set_threads(int32_t n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* Apply a given move (or ORC_NULL_MOVE) at iteration `it` to a CSR schedule in place
 * and update the tabu list (R6). */
int32_t orc_apply_tabu_move(const orc_instance *in, int32_t tenure, int32_t it, int32_t *off,
                            int32_t *route, int32_t *tabu_until, uint32_t id) {
  if (id == ORC_NULL_MOVE) return ORC_OK;
  int M = in->n_missions, V = in->n_vehicles;
  sched s, t;
  if (sched_alloc(&s, V, M) != ORC_OK || sched_alloc(&t, V, M) != ORC_OK) return ORC_E_NOMEM;
  int rc = sched_from_csr(&s, off, route);
  moved_t mv;
  if (rc == ORC_OK && !apply_move(in, &s, id, &t, &mv)) rc = ORC_E_INVALID;
  if (rc == ORC_OK) {
    for (int j = 0; j < mv.n; j++) tabu_until[(int64_t)mv.mission[j] * V + mv.from[j]] = it + tenure;
    sched_to_csr(&t, off, route);
  }
  sched_free(&s);
  sched_free(&t);
  return rc;
}

/* Algorithm 3 under readings R5-R7, from a given schedule (or from Algorithm 1 when
 * init_off is NULL), for a fixed number of iterations. Outputs the best schedule,
 * its objective and iteration (-1 = the initial schedule), and per iteration the
 * applied move id (ORC_NULL_MOVE when none) and the objective after it. */
int32_t orc_tabu_search(const orc_instance *in, int32_t tenure, int32_t iterations,
                        const int32_t *init_off, const int32_t *init_route,
                        int32_t *best_off, int32_t *best_route, int64_t *z_best_out,
                        int32_t *best_it_out, uint32_t *traj_move, int64_t *traj_z) {
  int rc = check_instance(in);
  if (rc != ORC_OK) return rc;
  int M = in->n_missions, V = in->n_vehicles;
  int32_t *off = (int32_t *)malloc(sizeof(int32_t) * (size_t)(V + 1));
  int32_t *route = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
  int32_t *tabu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1) * (size_t)V);
  int64_t n = orc_num_moves(M, V);
  int64_t *delta = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  uint32_t *ids = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  if (init_off) {
    memcpy(off, init_off, sizeof(int32_t) * (size_t)(V + 1));
    memcpy(route, init_route, sizeof(int32_t) * (size_t)M);
    if (!orc_feasible(in, off, route)) rc = ORC_E_INFEASIBLE_INIT;
  } else {
    rc = orc_greedy_init(in, off, route);
  }
  if (rc == ORC_OK) {
    for (int64_t i = 0; i < (int64_t)M * V; i++) tabu[i] = -1;
    int64_t z = orc_cost(in, off, route, NULL, NULL);
    int64_t z_best = z;
    int32_t best_it = -1;
    memcpy(best_off, off, sizeof(int32_t) * (size_t)(V + 1));
    memcpy(best_route, route, sizeof(int32_t) * (size_t)M);
    for (int it = 0; it < iterations && rc == ORC_OK; it++) {
      int64_t chosen = -1;
      int64_t got = orc_eval_neighbourhood(in, off, route, tabu, it, z_best, delta, NULL, ids, &chosen);
      if (got < 0) { rc = (int)got; break; }
      uint32_t id = chosen >= 0 ? ids[chosen] : ORC_NULL_MOVE;
      rc = orc_apply_tabu_move(in, tenure, it, off, route, tabu, id);
      z = orc_cost(in, off, route, NULL, NULL);
      if (traj_move) traj_move[it] = id;
      if (traj_z) traj_z[it] = z;
      if (z < z_best) {
        z_best = z;
        best_it = it;
        memcpy(best_off, off, sizeof(int32_t) * (size_t)(V + 1));
        memcpy(best_route, route, sizeof(int32_t) * (size_t)M);
      }
    }
    *z_best_out = z_best;
    *best_it_out = best_it;
  }
  free(off);
  free(route);
  free(tabu);
  free(delta);
  free(ids);
  return rc;
}

/* ------------------------------------------------------------------------------------
 * Algorithm 2 (Neighbourhood Search) and Algorithm 3 as printed (a per-mission sweep
 * with a tabu list), under these readings:
 *   S1  A sweep takes the vehicles i in a fixed order, 0..V-1 unless an order is given;
 *       the missions j tried for i are i's route as it stands when i's turn starts, in
 *       route order, or by increasing given rank. (During i's turn missions only leave
 *       i, each at most once, so this is well defined.) The two orders stand for the
 *       paper's random permutation vectors of the two outer loops, passed in, and stay
 *       the same for every sweep of the search. Trying one mission is one step; steps
 *       are counted from 0 over the whole search.
 *   S2  Candidates for j: every other vehicle k (index order) whose type may fly j
 *       (con9), and on k every insertion point q = 0..n_k in order (q = n_k appends).
 *       The first insertion point whose schedule is infeasible (duty cap in HARD mode,
 *       deadlines) ends the scan of k: the later points of k are not tried (the
 *       listings' "continue to the next base" inside the loop over positions).
 *   S3  Algorithm 2 applies the candidate with the least (delta, k, q) when its delta
 *       is negative (the best position starts as j's current one); sweeps repeat while
 *       a sweep applied a move, at most max_sweeps.
 *   S4  Algorithm 3: the tabu list holds pairs (mission, vehicle). A pair (j, k) whose
 *       counter has not run out takes base k out of j's scan (the listing's "continue
 *       to the next k"); there is no aspiration. As in S3 the least (delta, k, q) of the
 *       other candidates is applied only when delta < 0 (the text adds an entry to the
 *       list only for a move that improves); applying it at step s from vehicle i makes
 *       (j, i) tabu through step s + tenure. Sweeps repeat while a sweep applied a move,
 *       at most max_sweeps.
 *   S4b The listing alone also reads as applying the least admissible candidate even
 *       when delta >= 0 (CurrentMin starting empty). Option accept_worse takes that
 *       reading; sweeps then repeat while a sweep lowered the best objective.
 *   S5  The result is the best schedule met (the first to reach the least objective).
 *   Trace: one entry per step, the relocation id (j << 13) | y of the applied move (y
 *   the node j now precedes: a mission, or M + k at the end of route k) or 0xFFFFFFFF
 *   when nothing was applied, and the objective after the step.
 * ------------------------------------------------------------------------------------ */

/* A permutation of 0..n-1, or NULL. */
static int is_permutation(const int32_t *p, int n) {
  if (!p) return 1;
  char *seen = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
  int ok = seen != NULL;
  for (int k = 0; k < n && ok; k++) {
    if (p[k] < 0 || p[k] >= n || seen[p[k]]) ok = 0;
    else seen[p[k]] = 1;
  }
  free(seen);
  return ok;
}

static int sweep_search(const orc_instance *in, int use_tabu, int accept_worse, int32_t tenure,
                        int32_t max_sweeps, int repair, const int32_t *vorder, const int32_t *mrank,
                        const int32_t *init_off, const int32_t *init_route, int32_t *best_off,
                        int32_t *best_route, int64_t *z_best_out, int32_t *counts_out,
                        uint32_t *trace_move, int64_t *trace_z, int64_t trace_cap) {
  int rc = check_instance(in);
  if (rc != ORC_OK) return rc;
  int M = in->n_missions, V = in->n_vehicles;
  if (!is_permutation(vorder, V) || !is_permutation(mrank, M)) return ORC_E_INVALID;
  int32_t *off = (int32_t *)malloc(sizeof(int32_t) * (size_t)(V + 1));
  int32_t *route = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
  int64_t *tabu = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M > 0 ? M : 1) * (size_t)V);
  int32_t *snap = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
  sched s, t, best_t;
  if (!off || !route || !tabu || !snap || sched_alloc(&s, V, M) != ORC_OK ||
      sched_alloc(&t, V, M) != ORC_OK || sched_alloc(&best_t, V, M) != ORC_OK)
    return ORC_E_NOMEM;
  if (init_off) {
    memcpy(off, init_off, sizeof(int32_t) * (size_t)(V + 1));
    memcpy(route, init_route, sizeof(int32_t) * (size_t)M);
    if (sched_from_csr(&s, off, route) != ORC_OK || !orc_feasible(in, off, route))
      rc = ORC_E_INFEASIBLE_INIT;
  } else {
    rc = greedy_core(in, repair, vorder, mrank, off, route);
  }
  sweep_ctx c = {0};
  int64_t sweeps = 0, z_init = 0;
  if (rc == ORC_OK) {
    sched_from_csr(&s, off, route);
    for (int64_t x = 0; x < (int64_t)(M > 0 ? M : 1) * V; x++) tabu[x] = -1;
    c.use_tabu = use_tabu;
    c.accept_worse = accept_worse;
    c.tenure = tenure;
    c.tabu = tabu;
    c.best_step = -1;
    c.z = c.z_best = z_init = sched_cost(in, &s, NULL, NULL);
    c.best = &best_t;
    c.trace_move = trace_move;
    c.trace_z = trace_z;
    c.trace_cap = trace_cap;
    c.vorder = vorder;
    c.mrank = mrank;
    sched_copy(&best_t, &s);
    int go_on = 1;
    while (go_on && sweeps < max_sweeps) {
      int64_t z_best_before = c.z_best;
      int applied = sweep_pass(in, &s, &t, snap, &c);
      sweeps++;
      go_on = accept_worse ? (c.z_best < z_best_before) : applied;
    }
    sched_to_csr(&best_t, best_off, best_route);
  }
  z_best_out[0] = c.z_best;
  z_best_out[1] = z_init;
  z_best_out[2] = c.z;
  counts_out[0] = (int32_t)sweeps;
  counts_out[1] = (int32_t)c.n_moves;
  counts_out[2] = (int32_t)c.step;
  counts_out[3] = (int32_t)(rc == ORC_OK ? c.best_step : -1);
  free(off);
  free(route);
  free(tabu);
  free(snap);
  sched_free(&s);
  sched_free(&t);
  sched_free(&best_t);
  return rc;
}

/* Algorithm 2 (readings S1-S3, S5), started from Algorithm 1 (with the repair of R12
 * when `repair` is set) unless init_off / init_route give the start; vorder / mrank
 * give the loop orders of S1 (NULL: index and route order), each a permutation.
 * z_out[3] = {best, initial, final} objectives;
 * counts_out[4] = {sweeps, moves applied, steps, step of the best (-1: initial)}. */
int32_t orc_neighbourhood_search(const orc_instance *in, int32_t max_sweeps, int32_t repair,
                                 const int32_t *vorder, const int32_t *mrank, const int32_t *init_off,
                                 const int32_t *init_route, int32_t *best_off, int32_t *best_route,
                                 int64_t *z_out, int32_t *counts_out, uint32_t *trace_move,
                                 int64_t *trace_z, int64_t trace_cap) {
  return sweep_search(in, 0, 0, 0, max_sweeps, repair, vorder, mrank, init_off, init_route, best_off, best_route, z_out,
                      counts_out, trace_move, trace_z, trace_cap);
}

/* Algorithm 3 as printed (readings S1, S2, S4 or S4b, S5); outputs as above. */
int32_t orc_tabu_sweep(const orc_instance *in, int32_t tenure, int32_t max_sweeps, int32_t accept_worse,
                       int32_t repair, const int32_t *vorder, const int32_t *mrank, const int32_t *init_off,
                       const int32_t *init_route, int32_t *best_off, int32_t *best_route, int64_t *z_out,
                       int32_t *counts_out, uint32_t *trace_move, int64_t *trace_z, int64_t trace_cap) {
  return sweep_search(in, 1, accept_worse != 0, tenure, max_sweeps, repair, vorder, mrank, init_off, init_route, best_off, best_route, z_out,
                      counts_out, trace_move, trace_z, trace_cap);
}
