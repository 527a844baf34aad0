"""Independent, brute-force restatements of the paper's model used to pin the oracle.

Nothing here shares code with the oracle or the CUDA path. A schedule is a tuple of
per-vehicle mission tuples. The objective and the constraints are written from the
ILP of Section 3 in its arc form: a binary x_ijk per arc i -> j flown by vehicle
(base) k, where the nodes are missions and bases.
"""
from __future__ import annotations

import itertools

import numpy as np

HARD, PENALTY = 0, 1


def csr_to_routes(off, route, V):
    off = [int(x) for x in off]
    return tuple(tuple(int(x) for x in route[off[v]:off[v + 1]]) for v in range(V))


def routes_to_csr(routes):
    off = [0]
    flat = []
    for r in routes:
        flat.extend(r)
        off.append(len(flat))
    return np.array(off, dtype=np.int32), np.array(flat if flat else [0], dtype=np.int32)[:len(flat)]


def arcs(routes):
    """x_ijk = 1 arcs: ((kind, id), (kind, id), k) with kind 'b' (base of k) or 'm'."""
    out = []
    for k, r in enumerate(routes):
        if not r:
            continue
        nodes = [("b", k)] + [("m", m) for m in r] + [("b", k)]
        out.extend((u, w, k) for u, w in zip(nodes, nodes[1:]))
    return out


def _end(inst, node, k):
    return int(inst.veh_base[k]) if node[0] == "b" else int(inst.delivery[node[1]])


def _start(inst, node, k):
    return int(inst.veh_base[k]) if node[0] == "b" else int(inst.pickup[node[1]])


def flights(inst, routes):
    """Minutes flown per vehicle: every arc's leg plus every served mission's own leg."""
    V = len(routes)
    f = [0] * V
    for (u, w, k) in arcs(routes):
        layer = int(inst.veh_type[k])
        f[k] += int(inst.travel[layer, _end(inst, u, k), _start(inst, w, k)])
    for k, r in enumerate(routes):
        layer = int(inst.veh_type[k])
        for m in r:
            f[k] += int(inst.travel[layer, inst.pickup[m], inst.delivery[m]])
    return f


def objective(inst, routes, cap_mode, lam):
    f = flights(inst, routes)
    z = sum(f)
    if cap_mode == PENALTY:
        z += lam * sum(max(0, x - inst.duty_cap) for x in f)
    return z


def feasible(inst, routes, cap_mode):
    """con1-con11 of Section 3 checked on the arc form (con8 read as a sum)."""
    M = len(inst.pickup)
    V = len(routes)
    A = arcs(routes)
    # con1 / con2: one arc into and one out of every mission, over all vehicles.
    into = {m: 0 for m in range(M)}
    outof = {m: 0 for m in range(M)}
    for (u, w, k) in A:
        if w[0] == "m":
            into[w[1]] += 1
        if u[0] == "m":
            outof[u[1]] += 1
    if any(into[m] != 1 or outof[m] != 1 for m in range(M)):
        return False
    # con3 / con4 / con5: per vehicle, flow is conserved and each node is entered
    # and left at most once.
    for k in range(V):
        ins, outs = {}, {}
        for (u, w, kk) in A:
            if kk != k:
                continue
            ins[w] = ins.get(w, 0) + 1
            outs[u] = outs.get(u, 0) + 1
        nodes = set(ins) | set(outs)
        if any(ins.get(n, 0) != outs.get(n, 0) for n in nodes):
            return False
        if any(v > 1 for v in ins.values()) or any(v > 1 for v in outs.values()):
            return False
    # con11: arcs touching a base use the vehicle's own base only.
    for (u, w, k) in A:
        for n in (u, w):
            if n[0] == "b" and n[1] != k:
                return False
    # con10: MTZ order exists (u_i = position along the route).
    pos = {}
    for k, r in enumerate(routes):
        for i, m in enumerate(r):
            pos[m] = i + 1
    n = max(M, 1)
    for (u, w, k) in A:
        if u[0] == "m" and w[0] == "m":
            if pos[u[1]] - pos[w[1]] + n > n - 1:
                return False
    # con9: a heli-only mission never flies on a plane.
    if inst.heli_only is not None:
        for k, r in enumerate(routes):
            if int(inst.veh_type[k]) != 0 and any(int(inst.heli_only[m]) for m in r):
                return False
    # con6: duty cap (HARD mode only).
    if cap_mode == HARD and any(f > inst.duty_cap for f in flights(inst, routes)):
        return False
    # con7 / con8: arrive-by times, leaving each delivery at its own deadline.
    if inst.deadline is not None:
        for (u, w, k) in A:
            layer = int(inst.veh_type[k])
            dep = 0 if u[0] == "b" else int(inst.deadline[u[1]])
            leg = int(inst.travel[layer, _end(inst, u, k), _start(inst, w, k)])
            if w[0] == "m":
                own = int(inst.travel[layer, inst.pickup[w[1]], inst.delivery[w[1]]])
                if dep + leg + own > int(inst.deadline[w[1]]):
                    return False
            elif dep + leg > inst.horizon:
                return False
    return True


def all_schedules(M, V):
    """Every assignment of M missions to V ordered routes: M! * C(M+V-1, V-1) of them."""
    for perm in itertools.permutations(range(M)):
        for cuts in itertools.combinations_with_replacement(range(M + 1), V - 1):
            b = (0,) + cuts + (M,)
            yield tuple(perm[b[i]:b[i + 1]] for i in range(V))


def remove(routes, m):
    return tuple(tuple(x for x in r if x != m) for r in routes)


def vehicle_of(routes, m):
    for k, r in enumerate(routes):
        if m in r:
            return k
    raise KeyError(m)


def node_after(routes, m):
    """The node after mission m: the next mission id, or M + v at the end of route v."""
    M = sum(len(r) for r in routes)
    for k, r in enumerate(routes):
        if m in r:
            i = r.index(m)
            return r[i + 1] if i + 1 < len(r) else M + k
    raise KeyError(m)


def neighbours(routes, universe):
    """Characterise the neighbourhood without building moves.

    Relocations of m: the schedules S' != S that equal S once m is deleted from
    both. Swaps of m1 < m2: the schedules with the same route lengths that differ
    from S in exactly two places, holding m1 and m2 exchanged. Returns a list of
    (move id, S', moved [(mission, from, to)]) in no particular order.
    """
    M = sum(len(r) for r in routes)
    out = []
    for m in range(M):
        base = remove(routes, m)
        for s2 in universe:
            if s2 != routes and remove(s2, m) == base:
                y = node_after(s2, m)
                out.append(((m << 13) | y, s2, [(m, vehicle_of(routes, m), vehicle_of(s2, m))]))
    shape = tuple(len(r) for r in routes)
    flat = [x for r in routes for x in r]
    for s2 in universe:
        if tuple(len(r) for r in s2) != shape:
            continue
        f2 = [x for r in s2 for x in r]
        diff = [i for i in range(M) if flat[i] != f2[i]]
        if len(diff) == 2 and flat[diff[0]] == f2[diff[1]] and flat[diff[1]] == f2[diff[0]]:
            m1, m2 = sorted((flat[diff[0]], flat[diff[1]]))
            out.append(((1 << 31) | (m1 << 13) | m2, s2,
                        [(m1, vehicle_of(routes, m1), vehicle_of(s2, m1)),
                         (m2, vehicle_of(routes, m2), vehicle_of(s2, m2))]))
    return out


def tabu_step(inst, routes, universe, tabu_until, it, z_best, cap_mode, lam):
    """One iteration of the reading R5-R7, derived by brute force over the universe.

    Returns (chosen id or None, S' or routes, moved list)."""
    z0 = objective(inst, routes, cap_mode, lam)
    best = None
    for mid, s2, moved in neighbours(routes, universe):
        if not feasible(inst, s2, cap_mode):
            continue
        z1 = objective(inst, s2, cap_mode, lam)
        tabu = any(tabu_until.get((x, to), -1) >= it for (x, _, to) in moved)
        if tabu and not z1 < z_best:
            continue
        key = (z1 - z0, mid)
        if best is None or key < best[0]:
            best = (key, s2, moved)
    if best is None:
        return None, routes, []
    return best[0][1], best[1], best[2]
