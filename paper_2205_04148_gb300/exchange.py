"""Halo exchange between ranks that hold different tiles of one member.

The paper fills the halos of a tile from its neighbours with a point-to-point
exchange between ranks, rotating vectors across cube edges (Section V-C).  On
one GPU the library does this inside a kernel (fv3_halo_fill); when the tiles
of a member live on different devices, the same plan (fv3_halo_plan) splits by
tile owner: an entry whose source tile is local is a copy, one whose source
lives on another rank is a value that rank sends.  Both sides walk the plan in
its own order, so the values of a message need no index.

Fields are tensors [arrays][local tiles][levels][plane] in the library's plane
layout (arrays: 1 for a scalar, 2 for a vector pair: the x-face array, then the
y-face array); the tiles of a rank are its owned tiles in increasing order.
The messages go through torch.distributed point-to-point operations (gloo on
CPU tensors, NCCL on device tensors); a message that does not arrive within
the timeout raises ExchangeError instead of waiting for ever.
"""
from __future__ import annotations

import datetime

import numpy as np


class ExchangeError(RuntimeError):
    pass


class TileExchange:
    """The part of one member's halo plan that concerns `rank`.

    entries: the plan (dict of arrays dst, src, dst_tile, src_tile, sign,
    flags, as fv3.halo_plan returns); owner[t]: the rank holding tile t;
    nlev, plane: levels and elements per plane of the fields; vector: the
    plan is a vector-pair plan (flags choose the array)."""

    def __init__(self, entries, owner, rank, nlev, plane, vector=False):
        self.rank = rank
        self.owner = list(owner)
        self.tiles = [t for t in range(len(owner)) if owner[t] == rank]
        self.nlev, self.plane = nlev, plane
        self.arrays = 2 if vector else 1
        slot = {t: k for k, t in enumerate(self.tiles)}
        ntl = len(self.tiles)
        owner = np.asarray(owner)
        dst_t, src_t = entries["dst_tile"], entries["src_tile"]
        sign = entries["sign"]
        dst_a = (entries["flags"] & 1) if vector else np.zeros_like(sign)
        src_a = ((entries["flags"] >> 1) & 1) if vector else np.zeros_like(sign)
        lev = np.arange(nlev, dtype=np.int64) * plane

        def flat(arr, tiles, off):  # level-0 offsets -> [entries, levels] flat indices
            s = np.array([slot[int(t)] for t in tiles], dtype=np.int64)
            base = (arr * ntl + s) * nlev * plane + off
            return (base[:, None] + lev[None, :]).reshape(-1)

        mine_dst = owner[dst_t] == rank
        nan = mine_dst & (sign == 0)
        local = mine_dst & (sign != 0) & (owner[src_t] == rank)
        self.nan_dst = flat(dst_a[nan], dst_t[nan], entries["dst"][nan])
        self.local_src = flat(src_a[local], src_t[local], entries["src"][local])
        self.local_dst = flat(dst_a[local], dst_t[local], entries["dst"][local])
        self.local_sign = np.repeat(sign[local], nlev)
        self.recv, self.send = {}, {}
        for peer in sorted(set(owner.tolist()) - {rank}):
            r = mine_dst & (sign != 0) & (owner[src_t] == peer)
            if r.any():
                self.recv[peer] = flat(dst_a[r], dst_t[r], entries["dst"][r])
            s = (owner[dst_t] == peer) & (sign != 0) & (owner[src_t] == rank)
            if s.any():
                self.send[peer] = (flat(src_a[s], src_t[s], entries["src"][s]), np.repeat(sign[s], nlev))
        self._t = None

    def shape(self):
        return (self.arrays, len(self.tiles), self.nlev, self.plane)

    def _tensors(self, like):
        import torch
        dev = like.device
        idx = lambda a: torch.as_tensor(a, dtype=torch.long, device=dev)  # noqa: E731
        val = lambda a: torch.as_tensor(a, dtype=like.dtype, device=dev)  # noqa: E731
        self._t = {"nan": idx(self.nan_dst), "ls": idx(self.local_src), "ld": idx(self.local_dst),
                   "lsg": val(self.local_sign),
                   "recv": {p: idx(d) for p, d in self.recv.items()},
                   "send": {p: (idx(s), val(g)) for p, (s, g) in self.send.items()},
                   "dev": dev, "dtype": like.dtype}

    def run(self, buf, timeout_s=30.0, group=None):
        """Fill the halo slots of the local tiles of `buf` (a contiguous
        tensor of shape self.shape()): local copies, NaN for the slots with
        no value, and the values the owners of the other tiles send."""
        import torch
        import torch.distributed as dist
        if tuple(buf.shape) != self.shape() or not buf.is_contiguous():
            raise ValueError("need a contiguous tensor of shape %s" % (self.shape(),))
        if self._t is None or self._t["dev"] != buf.device or self._t["dtype"] != buf.dtype:
            self._tensors(buf)
        T = self._t
        flat = buf.view(-1)
        reqs = []
        inbox, outbox = {}, {}  # the messages stay referenced until their waits end
        for peer, (s, g) in T["send"].items():
            outbox[peer] = flat[s] * g
            reqs.append((peer, dist.isend(outbox[peer], peer, group=group)))
        for peer, d in T["recv"].items():
            inbox[peer] = torch.empty(d.numel(), dtype=buf.dtype, device=buf.device)
            reqs.append((peer, dist.irecv(inbox[peer], peer, group=group)))
        if T["ls"].numel():
            flat[T["ld"]] = flat[T["ls"]] * T["lsg"]
        if T["nan"].numel():
            flat[T["nan"]] = float("nan")
        limit = datetime.timedelta(seconds=timeout_s)
        for peer, r in reqs:
            try:
                ok = r.wait(timeout=limit)
            except RuntimeError as e:
                raise ExchangeError("halo exchange with rank %d failed: %s" % (peer, e)) from e
            if ok is False:
                raise ExchangeError("halo exchange with rank %d: no message within %.1f s" % (peer, timeout_s))
        for peer, d in T["recv"].items():
            flat[d] = inbox[peer]
        return buf
