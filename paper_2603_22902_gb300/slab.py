"""Host-side schedule of the y-slab decomposition (argument marshalling and ordering
only: the step, the packing and the unpacking of the halo messages and the band sums
run in liblbm_gb300.so, see lbm_slab_* in include/lbm.h).

A lattice of ny rows is cut into bands; band k holds rows [y0_k, y1_k).  After every
step, each cut is crossed by two messages per direction (phase 1: the populations pushed
across it; phase 2: the boundary row's stencil inputs).  Per phase the order is fixed:
every band packs all its cut sides, the messages travel, every band unpacks.  The
transfers of one phase go in two passes, first every band's y-max message to the band
above (unpacked there on its y-min side), then every band's y-min message to the band
below, so that two ranks that are each other's upper and lower neighbour (two bands of a
periodic lattice) post their sends and receives in the same order.

Two transports:
  * LocalExchange: all bands in one process (one GPU): the message of the sender is the
    receive buffer of the receiver, so a transfer is no copy at all;
  * DistExchange: one band per rank, torch.distributed point-to-point (NCCL between GPUs,
    gloo on CPU for the tests); remote messages land in local buffers.
The diagnostics sums of the bands combine by a sum of the N volumes, the N solid
volumes and the non-finite counts and a maximum of the deviation max |sum phi - 1|.

Overlap (step(n, overlap=True)): a band's step splits into its inner tile rows, which
neither read nor write the rows the exchange touches, and its edge rows
(lbm_slab_step_part).  Per step: the inner rows of every band, then the exchange of the
previous step, then the edge rows; with `streams=(compute, exchange)` the exchange runs
on the second stream, after an event recorded behind the previous edge part, while the
inner part runs on the first, which waits for the exchange before the edge part.  The
last step's exchange follows the loop, so the bands end in the state of step(n).
"""
from __future__ import annotations

YMIN, YMAX = 2, 3
INNER, EDGE = 1, 2      # the parts of lbm_slab_step_part


def split_rows(ny: int, nbands: int):
    """Bands [y0, y1) of nearly equal height covering rows 0 .. ny - 1."""
    if not 1 <= nbands <= ny:
        raise ValueError("need 1 <= nbands <= ny")
    cuts = [round(k * ny / nbands) for k in range(nbands + 1)]
    return [(cuts[k], cuts[k + 1]) for k in range(nbands)]


def neighbours(k: int, nbands: int, periodic: bool):
    """(band below, band above) of band k, None where the band meets a global side."""
    below = k - 1 if k > 0 else (nbands - 1 if periodic and nbands > 1 else None)
    above = k + 1 if k < nbands - 1 else (0 if periodic and nbands > 1 else None)
    return below, above


def combine_sums(parts, N):
    """Diagnostics of the lattice from the sums of its bands (lbm_slab_sums)."""
    out = dict(mass=[0.0] * N, solid=[0.0] * N, max_sum_dev=0.0, nonfinite=0)
    for d in parts:
        for p in range(N):
            out["mass"][p] += d["mass"][p]
            out["solid"][p] += d["solid"][p]
        out["max_sum_dev"] = max(out["max_sum_dev"], d["max_sum_dev"])
        out["nonfinite"] += d["nonfinite"]
    return out


def _exchange_after(bands, exchange, streams, ev_edge):
    """One exchange; with streams, on the exchange stream after ev_edge, and the compute
    stream made to wait for it."""
    if streams is None:
        exchange()
        return
    import torch
    compute, xs = streams
    xs.wait_event(ev_edge)
    for b in bands:
        b.set_stream(xs)
    with torch.cuda.stream(xs):
        exchange()
    for b in bands:
        b.set_stream(compute)
    compute.wait_event(xs.record_event())


def overlapped_steps(bands, exchange, n, streams=None):
    """n steps of the bands with each exchange placed between the inner and the edge part
    of the next step (see the module's description); ends with the last step's exchange."""
    ev_edge = None
    for t in range(n):
        for b in bands:
            b.step_part(INNER)
        if t > 0:
            _exchange_after(bands, exchange, streams, ev_edge)
        for b in bands:
            b.step_part(EDGE)
        if streams is not None:
            ev_edge = streams[0].record_event()
    if n > 0:
        _exchange_after(bands, exchange, streams, ev_edge)


class LocalExchange:
    """Bands of one lattice in one process.  `bands` are objects with step(n),
    pack(side, phase, msg), unpack(side, phase, msg) and msg_bytes[phase] (SlabSolver);
    `alloc(nbytes)` returns a message buffer."""

    def __init__(self, bands, periodic, alloc):
        self.bands = list(bands)
        n = len(self.bands)
        self.links = []          # (sender, sender side, receiver, receiver side)
        for k in range(n):
            below, above = neighbours(k, n, periodic)
            if above is not None:
                self.links.append((k, YMAX, above, YMIN))
            if below is not None:
                self.links.append((k, YMIN, below, YMAX))
        self.msg = {(k, side, ph): alloc(self.bands[k].msg_bytes[ph])
                    for (k, side, _, _) in self.links for ph in (1, 2)}

    def exchange(self):
        for ph in (1, 2):
            for k, side, _, _ in self.links:
                self.bands[k].pack(side, ph, self.msg[(k, side, ph)])
            for k, side, r, rside in self.links:
                self.bands[r].unpack(rside, ph, self.msg[(k, side, ph)])

    def step(self, n=1, overlap=False, streams=None):
        if overlap:
            overlapped_steps(self.bands, self.exchange, n, streams)
            return
        for _ in range(n):
            for b in self.bands:
                b.step(1)
            self.exchange()

    def sums(self, N):
        return combine_sums([b.sums() for b in self.bands], N)


class DistExchange:
    """One band per rank of a torch.distributed group (rank k holds band k).  `alloc`
    gives the message buffers that pack and unpack use; with `host_alloc` (a backend that
    moves host memory only, e.g. gloo) the messages travel through host buffers of that
    size, copied to and from the message buffers on the current stream."""

    def __init__(self, band, periodic, alloc, dist=None, host_alloc=None):
        if dist is None:
            import torch.distributed as dist
        self.dist = dist
        self.band = band
        self.rank, n = dist.get_rank(), dist.get_world_size()
        self.below, self.above = neighbours(self.rank, n, periodic)
        self.send = {(side, ph): alloc(band.msg_bytes[ph]) for side in (YMIN, YMAX) for ph in (1, 2)}
        self.recv = {(side, ph): alloc(band.msg_bytes[ph]) for side in (YMIN, YMAX) for ph in (1, 2)}
        self.host_send = self.host_recv = None
        if host_alloc is not None:
            self.host_send = {k: host_alloc(band.msg_bytes[k[1]]) for k in self.send}
            self.host_recv = {k: host_alloc(band.msg_bytes[k[1]]) for k in self.recv}

    def _transfer(self, ph):
        """Pass 1: y-max messages go up (received on the y-min side); pass 2: y-min
        messages go down (received on the y-max side).  Each pass is one batch of
        point-to-point operations, posted in the same order on every rank."""
        d = self.dist
        staged = self.host_send is not None
        sbuf = self.host_send if staged else self.send
        rbuf = self.host_recv if staged else self.recv
        for send_side, peer_send, recv_side, peer_recv in ((YMAX, self.above, YMIN, self.below),
                                                          (YMIN, self.below, YMAX, self.above)):
            ops = []
            if peer_send is not None:
                if staged:
                    sbuf[(send_side, ph)].copy_(self.send[(send_side, ph)])
                ops.append(d.P2POp(d.isend, sbuf[(send_side, ph)], peer_send, tag=10 * ph + send_side))
            if peer_recv is not None:
                ops.append(d.P2POp(d.irecv, rbuf[(recv_side, ph)], peer_recv, tag=10 * ph + (5 - recv_side)))
            if ops:
                for req in d.batch_isend_irecv(ops):
                    req.wait()
            if staged and peer_recv is not None:
                self.recv[(recv_side, ph)].copy_(rbuf[(recv_side, ph)])

    def exchange(self):
        b = self.band
        sides = [s for s, peer in ((YMIN, self.below), (YMAX, self.above)) if peer is not None]
        for ph in (1, 2):
            for side in sides:
                b.pack(side, ph, self.send[(side, ph)])
            self._transfer(ph)
            for side in sides:
                b.unpack(side, ph, self.recv[(side, ph)])

    def step(self, n=1, overlap=False, streams=None):
        if overlap:
            overlapped_steps([self.band], self.exchange, n, streams)
            return
        for _ in range(n):
            self.band.step(1)
            self.exchange()

    def sums(self, N):
        """Lattice diagnostics: all-reduce of the band sums (sum, and max of the deviation)."""
        import torch
        d = self.band.sums()
        t = torch.tensor(d["mass"] + d["solid"] + [float(d["nonfinite"])], dtype=torch.float64)
        m = torch.tensor([d["max_sum_dev"]], dtype=torch.float64)
        dev = getattr(self.band, "reduce_device", "cpu")
        t, m = t.to(dev), m.to(dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        self.dist.all_reduce(m, op=self.dist.ReduceOp.MAX)
        t, m = t.cpu().tolist(), float(m.cpu().item())
        return dict(mass=t[:N], solid=t[N:2 * N], max_sum_dev=m, nonfinite=int(round(t[2 * N])))
