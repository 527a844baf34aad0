"""Continuous-batching request server over asched_serve (host side).

The device side is one persistent launch (asched_serve): every CTA takes the next
published request as soon as it is free. Optionally a second persistent launch made of
thread-block clusters takes the largest requests (at least `big_missions` missions), each
solved by a whole cluster, so that they do not set the tail latency; it is launched
first, while the device is idle, and the one-CTA launch takes the remaining SMs. This module owns the host side: a fixed pool
of device-resident request slots sized by a device-memory budget, admission of new
requests into free slots while others are running, publication by copies ordered on a
dedicated stream, and completion polling. All device memory and pinned staging is
allocated up front, so nothing allocates (or implicitly synchronises) while the
persistent launch runs; all work goes to non-blocking streams.
"""
from __future__ import annotations

import ctypes
import time
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import CTRL_LEN, CTRL_PUBLISHED, CTRL_SERVED, CTRL_STARTED, CTRL_STOP, SLOT_HEADER
from .api import INFO_LEN, _ptr


class Server:
    """A request server for instances up to (max_loc, max_vehicles, max_missions).

    n_slots is the number of requests that can be resident at once; it is further
    limited so that the slots fit budget_bytes of device memory."""

    def __init__(self, max_loc: int, max_vehicles: int, max_missions: int, n_types: int = 1,
                 n_slots: int = 1024, has_deadlines: bool = False, budget_bytes: int = 40 << 30,
                 device="cuda", big_missions: Optional[int] = None, big_cluster: int = 16,
                 big_clusters: int = 1):
        self.device = torch.device(device)
        self.Lc, self.Vc, self.Mc, self.nt = int(max_loc), int(max_vehicles), int(max_missions), int(n_types)
        sw, ow = ctypes.c_int32(0), ctypes.c_int32(0)
        _lib.check(_lib.load().asched_server_sizes(self.Lc, self.Vc, self.Mc, self.nt,
                                                   ctypes.byref(sw), ctypes.byref(ow)),
                   "asched_server_sizes")
        self.slot_words, self.out_words = sw.value, ow.value
        per_slot = 4 * (self.slot_words + self.out_words + 1)
        self.slot_bytes = per_slot
        self.n_slots = int(max(1, min(n_slots, budget_bytes // per_slot)))
        self.ring_len = 4 * self.n_slots
        self.has_deadlines = bool(has_deadlines)
        dev = self.device
        self.slot_data = torch.zeros(self.n_slots * self.slot_words, dtype=torch.int32, device=dev)
        self.slot_out = torch.zeros(self.n_slots * self.out_words, dtype=torch.int32, device=dev)
        self.ring = torch.zeros(self.ring_len, dtype=torch.int32, device=dev)
        self.control = torch.zeros(CTRL_LEN, dtype=torch.int32, device=dev)
        self.done = torch.full((self.n_slots,), -1, dtype=torch.int32, device=dev)
        # pinned staging (each entry is rewritten only after its copy has completed)
        self.stage = torch.zeros((self.n_slots, self.slot_words), dtype=torch.int32).pin_memory()
        self.ring_stage = torch.zeros(self.ring_len, dtype=torch.int32).pin_memory()
        self.pub_stage = torch.zeros(self.ring_len, dtype=torch.int32).pin_memory()
        self.stop_stage = torch.ones(1, dtype=torch.int32).pin_memory()
        self.done_host = torch.full((self.n_slots,), -1, dtype=torch.int32).pin_memory()
        self.out_host = torch.zeros(self.out_words, dtype=torch.int32).pin_memory()
        # control words are read into this pinned buffer: an allocation of pinned memory
        # while a persistent launch runs could wait for the launch to end
        self.ctrl_host = torch.zeros(CTRL_LEN, dtype=torch.int32).pin_memory()
        self._stage_np = self.stage.numpy()
        self._ring_np = self.ring_stage.numpy()
        self._pub_np = self.pub_stage.numpy()
        self._done_np = self.done_host.numpy()
        self.serve_stream = torch.cuda.Stream(device=dev)
        self.copy_stream = torch.cuda.Stream(device=dev)
        self.poll_stream = torch.cuda.Stream(device=dev)
        self.free = list(range(self.n_slots - 1, -1, -1))
        self.slot_seq = np.full(self.n_slots, -1, np.int64)
        self.next_ticket = 0
        self.running = False
        self.struct = _lib.Server(self.n_slots, self.ring_len, self.Lc, self.Vc, self.Mc, self.nt,
                                  int(self.has_deadlines), _ptr(self.slot_data), _ptr(self.slot_out),
                                  _ptr(self.ring), _ptr(self.control), _ptr(self.done))
        # the large-request lane: its own ring, control words, stream and ticket counter
        self.big_missions = None if big_missions is None else int(big_missions)
        self.big_cluster, self.big_clusters = int(big_cluster), int(big_clusters)
        self.big_ctas = 0
        if self.big_missions is not None:
            self.ring_big = torch.zeros(self.ring_len, dtype=torch.int32, device=dev)
            self.control_big = torch.zeros(CTRL_LEN, dtype=torch.int32, device=dev)
            self.ring_stage_big = torch.zeros(self.ring_len, dtype=torch.int32).pin_memory()
            self.pub_stage_big = torch.zeros(self.ring_len, dtype=torch.int32).pin_memory()
            self._ring_big_np = self.ring_stage_big.numpy()
            self._pub_big_np = self.pub_stage_big.numpy()
            self.big_stream = torch.cuda.Stream(device=dev)
            self.next_ticket_big = 0
            self.struct_big = _lib.Server(self.n_slots, self.ring_len, self.Lc, self.Vc, self.Mc, self.nt,
                                          int(self.has_deadlines), _ptr(self.slot_data), _ptr(self.slot_out),
                                          _ptr(self.ring_big), _ptr(self.control_big), _ptr(self.done))

    # ------------------------------------------------------------------ lifecycle
    def _read_control(self, control, k: int) -> int:
        with torch.cuda.stream(self.poll_stream):
            self.ctrl_host[k:k + 1].copy_(control[k:k + 1], non_blocking=True)
        self.poll_stream.synchronize()
        return int(self.ctrl_host[k].item())

    def start(self, params: _lib.Params, idle_timeout_s: float = 10.0, max_ctas: int = 0):
        torch.cuda.synchronize(self.device)  # buffers are initialised
        L = _lib.load()
        sms = torch.cuda.get_device_properties(self.device).multi_processor_count
        if self.big_missions is not None:
            big = _lib.Params(params.tenure, params.iterations, params.cap_mode, params.lam,
                              self.big_cluster, params.block_threads, params.timeout_ns, params.flags)
            want = self.big_cluster * self.big_clusters
            _lib.check(L.asched_serve(ctypes.byref(self.struct_big), ctypes.byref(big), int(idle_timeout_s * 1e9),
                                      want, ctypes.c_void_p(self.big_stream.cuda_stream)), "asched_serve (clusters)")
            # the clusters must be resident before the one-CTA launch fills the device
            t0 = time.perf_counter()
            while self._read_control(self.control_big, CTRL_STARTED) < want:
                if time.perf_counter() - t0 > 5.0:
                    raise RuntimeError("the cluster launch did not start")
                time.sleep(1e-3)
            self.big_ctas = want
        rest = (max_ctas if max_ctas > 0 else sms) - self.big_ctas
        rc = L.asched_serve(ctypes.byref(self.struct), ctypes.byref(params), int(idle_timeout_s * 1e9),
                            int(max(rest, 1)), ctypes.c_void_p(self.serve_stream.cuda_stream))
        _lib.check(rc, "asched_serve")
        self.running = True

    def stop(self):
        """Ask the launch to end once every published request is taken; wait for it."""
        if not self.running:
            return
        with torch.cuda.stream(self.copy_stream):
            self.control[CTRL_STOP:CTRL_STOP + 1].copy_(self.stop_stage, non_blocking=True)
            if self.big_missions is not None:
                self.control_big[CTRL_STOP:CTRL_STOP + 1].copy_(self.stop_stage, non_blocking=True)
        self.serve_stream.synchronize()
        if self.big_missions is not None:
            self.big_stream.synchronize()
        self.running = False

    # ------------------------------------------------------------------ requests
    def pack(self, slot: int, inst, seq: int):
        """Write an instance into the pinned staging row of a slot."""
        L, V, M = int(inst.travel.shape[1]), len(inst.veh_base), len(inst.pickup)
        if int(inst.travel.shape[0]) != self.nt or L > self.Lc or V > self.Vc or M > self.Mc:
            raise ValueError("instance exceeds the server's slot capacity")
        if (inst.deadline is not None) != self.has_deadlines:
            raise ValueError("deadlines must match the server's has_deadlines")
        row = self._stage_np[slot]
        flags = (1 if inst.heli_only is not None else 0) | (2 if inst.deadline is not None else 0)
        row[:SLOT_HEADER] = 0
        row[0:7] = (L, V, M, int(inst.duty_cap), int(inst.horizon), flags, seq)
        o = SLOT_HEADER
        row[o:o + self.nt * L * L] = np.asarray(inst.travel, np.int32).reshape(-1)
        o = SLOT_HEADER + self.nt * self.Lc * self.Lc
        row[o:o + V] = inst.veh_base
        row[o + self.Vc:o + self.Vc + V] = inst.veh_type
        o += 2 * self.Vc
        row[o:o + M] = inst.pickup
        row[o + self.Mc:o + self.Mc + M] = inst.delivery
        if inst.heli_only is not None:
            row[o + 2 * self.Mc:o + 2 * self.Mc + M] = inst.heli_only
        if inst.deadline is not None:
            row[o + 3 * self.Mc:o + 3 * self.Mc + M] = inst.deadline
        return o + 4 * self.Mc

    def submit(self, inst, seq: int) -> Optional[int]:
        """Admit a request into a free slot and publish it; None if every slot is busy."""
        if not self.free:
            return None
        slot = self.free.pop()
        used = self.pack(slot, inst, seq)
        big = self.big_missions is not None and len(inst.pickup) >= self.big_missions
        if big:
            t, ring, control = self.next_ticket_big, self.ring_big, self.control_big
            ring_stage, pub_stage, ring_np, pub_np = (self.ring_stage_big, self.pub_stage_big,
                                                      self._ring_big_np, self._pub_big_np)
        else:
            t, ring, control = self.next_ticket, self.ring, self.control
            ring_stage, pub_stage, ring_np, pub_np = self.ring_stage, self.pub_stage, self._ring_np, self._pub_np
        r = t % self.ring_len
        ring_np[r] = slot
        pub_np[r] = t + 1
        self.slot_seq[slot] = seq
        base = slot * self.slot_words
        with torch.cuda.stream(self.copy_stream):
            self.slot_data[base:base + used].copy_(self.stage[slot, :used], non_blocking=True)
            ring[r:r + 1].copy_(ring_stage[r:r + 1], non_blocking=True)
            control[CTRL_PUBLISHED:CTRL_PUBLISHED + 1].copy_(pub_stage[r:r + 1], non_blocking=True)
        if big:
            self.next_ticket_big = t + 1
        else:
            self.next_ticket = t + 1
        return slot

    def poll(self):
        """Completed requests since the last poll: list of (slot, seq). Their slots are
        free again; read results with result() before the slot is reused."""
        with torch.cuda.stream(self.poll_stream):
            self.done_host.copy_(self.done, non_blocking=True)
        self.poll_stream.synchronize()
        busy = self.slot_seq >= 0
        hit = np.nonzero(busy & (self._done_np == self.slot_seq.astype(np.int32)))[0]
        out = []
        for s in hit:
            out.append((int(s), int(self.slot_seq[s])))
            self.slot_seq[s] = -1
            self.free.append(int(s))
        return out

    def result(self, slot: int):
        """Copy one slot's outputs to the host (synchronous on the poll stream)."""
        o = slot * self.out_words
        with torch.cuda.stream(self.poll_stream):
            self.out_host.copy_(self.slot_out[o:o + self.out_words], non_blocking=True)
        self.poll_stream.synchronize()
        w = self.out_host.numpy()
        Vc, Mc = self.Vc, self.Mc
        return {"route_off": w[:Vc + 1].copy(), "route": w[Vc + 1:Vc + 1 + Mc].copy(),
                "flight": w[Vc + 1 + Mc:2 * Vc + 1 + Mc].copy(),
                "overflow": w[2 * Vc + 1 + Mc:3 * Vc + 1 + Mc].copy(),
                "info": w[3 * Vc + 1 + Mc:3 * Vc + 1 + Mc + INFO_LEN].copy()}

    def served(self) -> int:
        n = self._read_control(self.control, CTRL_SERVED)
        if self.big_missions is not None:
            n += self._read_control(self.control_big, CTRL_SERVED)
        return n


def run_stream(server: Server, requests, arrivals_s, on_done=None, poll_interval_s: float = 50e-6,
               stall_timeout_s: float = 30.0):
    """Feed requests at their arrival times (seconds from now) into a started server and
    wait for all of them. Returns per-request latency in seconds (arrival -> completion
    observed by the host) and the wall time. on_done(i, slot) may read results. Raises
    if requests are pending and none completes for stall_timeout_s (a launch that ended,
    for instance after its idle timeout, serves nothing more)."""
    n = len(requests)
    lat = np.zeros(n)
    slot_of = {}
    pending = 0
    i = 0
    t0 = time.perf_counter()
    seq_to_req = {}
    completed = 0
    last_progress = time.perf_counter()
    while completed < n:
        now = time.perf_counter() - t0
        while i < n and arrivals_s[i] <= now:
            slot = server.submit(requests[i], i)
            if slot is None:
                break  # every slot is busy: admit later
            seq_to_req[i] = i
            slot_of[i] = slot
            i += 1
            pending += 1
        if pending:
            for slot, seq in server.poll():
                lat[seq] = time.perf_counter() - t0 - arrivals_s[seq]
                if on_done is not None:
                    on_done(seq, slot)
                pending -= 1
                completed += 1
                last_progress = time.perf_counter()
            if time.perf_counter() - last_progress > stall_timeout_s:
                raise RuntimeError(f"{pending} requests pending and none completed for {stall_timeout_s:g} s")
        else:
            last_progress = time.perf_counter()
        if i < n and not pending:
            wait = arrivals_s[i] - (time.perf_counter() - t0)
            if wait > 2 * poll_interval_s:
                time.sleep(wait - poll_interval_s)
    return lat, time.perf_counter() - t0
