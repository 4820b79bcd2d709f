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
An exchange is three steps: pack (each peer's message gathered with the
vector sign), local (halo slots filled from the rank's own tiles, NaN where
the plan has no value) and unpack (each received message scattered into its
halo slots).  On device tensors every step runs in the library's kernels
(fv3_halo_gather, fv3_halo_copy, fv3_halo_scatter); on CPU tensors in torch.
The messages go through torch.distributed point-to-point operations.  With
gloo and CPU tensors a message that does not arrive within the timeout
raises ExchangeError instead of waiting for ever.  With NCCL and device
tensors the timeout bounds only the host's wait: a peer that never sends
can leave the receive waiting on the device, so that case has no failure
guarantee; the device path has been checked on one GPU only (pack and
unpack against fv3_halo_fill), not between GPUs.
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

        # halo slots are filled from interior values only: no source slot of
        # the plan is also a destination, so the steps of an exchange (and
        # the entries within a step) do not depend on their order
        dst_key = set(zip(dst_t.tolist(), dst_a.tolist(), entries["dst"].tolist()))
        src_key = set(zip(src_t[sign != 0].tolist(), src_a[sign != 0].tolist(), entries["src"][sign != 0].tolist()))
        if dst_key & src_key:
            raise ValueError("plan reads a slot that it also writes")
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
        if dev.type == "cuda":   # the kernels take the signs as int8
            val = lambda a: torch.as_tensor(a, dtype=torch.int8, device=dev)  # noqa: E731
        else:
            val = lambda a: torch.as_tensor(a, dtype=like.dtype, device=dev)  # noqa: E731
        self._t = {"nan": idx(self.nan_dst), "ls": idx(self.local_src), "ld": idx(self.local_dst),
                   "lsg": val(self.local_sign),
                   "recv": {p: idx(d) for p, d in self.recv.items()},
                   "send": {p: (idx(s), val(g)) for p, (s, g) in self.send.items()},
                   "dev": dev, "dtype": like.dtype}

    def _check(self, buf):
        if tuple(buf.shape) != self.shape() or not buf.is_contiguous():
            raise ValueError("need a contiguous tensor of shape %s" % (self.shape(),))
        if self._t is None or self._t["dev"] != buf.device or self._t["dtype"] != buf.dtype:
            self._tensors(buf)
        return self._t

    def pack(self, buf):
        """{peer: message}: the values of `buf` each peer needs, in plan order,
        with the vector sign applied"""
        T = self._check(buf)
        flat = buf.view(-1)
        if buf.is_cuda:
            from . import fv3
            return {p: fv3.halo_gather(flat, s, g) for p, (s, g) in T["send"].items()}
        return {p: flat[s] * g for p, (s, g) in T["send"].items()}

    def local(self, buf):
        """halo slots filled from the rank's own tiles, NaN where the plan has
        no value"""
        T = self._check(buf)
        flat = buf.view(-1)
        if buf.is_cuda:
            from . import fv3
            if T["ls"].numel():
                fv3.halo_copy(flat, T["ls"], T["ld"], T["lsg"])
            if T["nan"].numel():
                fv3.halo_scatter(flat, T["nan"])
            return buf
        if T["ls"].numel():
            flat[T["ld"]] = flat[T["ls"]] * T["lsg"]
        if T["nan"].numel():
            flat[T["nan"]] = float("nan")
        return buf

    def unpack(self, buf, peer, message):
        """the message of `peer` into its halo slots"""
        T = self._check(buf)
        d = T["recv"][peer]
        if message.numel() != d.numel():
            raise ExchangeError("message of rank %d has %d values, the plan %d" % (peer, message.numel(), d.numel()))
        flat = buf.view(-1)
        if buf.is_cuda:
            from . import fv3
            fv3.halo_scatter(flat, d, message.contiguous())
        else:
            flat[d] = message
        return buf

    def run(self, buf, timeout_s=30.0, group=None):
        """Fill the halo slots of the local tiles of `buf` (a contiguous
        tensor of shape self.shape()): local copies, NaN for the slots with
        no value, and the values the owners of the other tiles send."""
        import torch
        import torch.distributed as dist
        T = self._check(buf)
        reqs = []
        inbox = {}
        outbox = self.pack(buf)   # the messages stay referenced until their waits end
        for peer, msg in outbox.items():
            reqs.append((peer, dist.isend(msg, peer, group=group)))
        for peer, d in T["recv"].items():
            inbox[peer] = torch.empty(d.numel(), dtype=buf.dtype, device=buf.device)
            reqs.append((peer, dist.irecv(inbox[peer], peer, group=group)))
        self.local(buf)
        limit = datetime.timedelta(seconds=timeout_s)
        for peer, r in reqs:
            try:
                ok = r.wait(timeout=limit)
            except RuntimeError as e:
                raise ExchangeError("halo exchange with rank %d failed: %s" % (peer, e)) from e
            if ok is False:
                raise ExchangeError("halo exchange with rank %d: no message within %.1f s" % (peer, timeout_s))
        for peer in T["recv"]:
            self.unpack(buf, peer, inbox[peer])
        return buf
