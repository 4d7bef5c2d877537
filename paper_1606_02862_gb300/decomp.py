"""Domain decomposition of one periodic box into z slabs (Sec. 2.1: the
simulation domain is divided into local domains made of supercells, one per
device; Sec. 1: the code runs on many GPUs).

Each slab is a one-box subdomain context (pic_set_subdomain).  Per step it
exchanges with its two neighbours on a ring (periodic in z):

  PUSH      -> J guard planes (added into the neighbour's interior) and the
               particles that left through a z face (migrants)
  FRAMES
  B_FIRST   -> B planes (the neighbour's guards)
  E         -> E planes
  B_SECOND  -> B planes

so the slabs together take exactly the steps of the undivided box.  The
messages are device buffers of fixed size (no host round trip for counts):
the caller's transport moves them -- NCCL point-to-point between processes
(one GPU each), or device copies between slabs held by one process.

The slab objects only need the calls below (libpic contexts through
LibpicSlab; a test can stand any other implementation of the same step in
for them):
    step_stage(stage); halo_floats(which, side); halo_pack(which, side, buf);
    halo_unpack(which, side, buf); migrant_bytes(); migrants_pack(side, buf);
    migrants_accept(side, buf)
"""
from __future__ import annotations

from dataclasses import dataclass

from . import pic

FIELDS = (pic.FIELD_E, pic.FIELD_B, pic.FIELD_J)
MIGRANTS = "migrants"


@dataclass(frozen=True)
class SlabLayout:
    """z planes of each of `world` slabs of a box nz planes high, in whole
    supercell rows of LZ planes, as even as the rows allow (the first
    nrows % world slabs get one row more)."""
    nz: int
    world: int
    LZ: int

    def __post_init__(self):
        if self.nz % self.LZ:
            raise ValueError("nz must be a multiple of the supercell edge LZ")
        if self.rows < self.world:
            raise ValueError("fewer supercell rows than slabs")
        if min(self.extent(r)[1] for r in range(self.world)) < 4:
            raise ValueError("a slab needs at least 4 planes")

    @property
    def rows(self):
        return self.nz // self.LZ

    def extent(self, rank):
        """(z0, nz_local) of slab `rank`."""
        q, r = divmod(self.rows, self.world)
        rows = q + (1 if rank < r else 0)
        z0 = (rank * q + min(rank, r)) * self.LZ
        return z0, rows * self.LZ

    def owner(self, z):
        """Slab index of every global z coordinate (numpy array)."""
        import numpy as np

        starts = np.array([self.extent(r)[0] for r in range(self.world)] + [self.nz])
        return np.searchsorted(starts, np.mod(z, self.nz), side="right") - 1


def split_particles(layout: SlabLayout, rank, x, u, w):
    """The particles of slab `rank` in its local coordinates (z - z0)."""
    import numpy as np

    x = np.asarray(x, dtype=np.float64)
    z = np.mod(x[:, 2], layout.nz)
    sel = layout.owner(z) == rank
    z0, _ = layout.extent(rank)
    xl = x[sel].copy()
    xl[:, 2] = z[sel] - z0
    return xl, np.asarray(u)[sel], None if w is None else np.asarray(w)[sel]


# ------------------------------------------------------------------ transports

class LocalRing:
    """Every slab of the ring in this process: the message of slab p to its
    upper neighbour arrives as the lower message of slab p + 1 (and the
    reverse), by a device (or host) copy on the current stream."""

    def __init__(self, nslabs):
        self.n = nslabs

    def positions(self):
        return list(range(self.n))

    def swap(self, send, recv):
        """send[p][side] -> recv[(p +- 1) % n][1 - side]."""
        for p in range(self.n):
            recv[(p + 1) % self.n][0].copy_(send[p][1])
            recv[(p - 1) % self.n][1].copy_(send[p][0])


class DistRing:
    """One slab per process (rank = ring position) over torch.distributed
    point-to-point: NCCL for device buffers, gloo for host buffers.  Both
    messages are posted as one batch, sends before receives, in the same
    order on every rank, so that with two ranks (the neighbour below is the
    one above) the pairs still match in order; tags tell them apart where
    the backend uses tags."""

    def __init__(self, dist, group=None):
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def positions(self):
        return [self.rank]

    def swap(self, send, recv):
        me = self.rank
        if self.world == 1:
            LocalRing(1).swap(send, recv)
            return
        up, dn = (me + 1) % self.world, (me - 1) % self.world
        d = self.dist
        ops = [d.P2POp(d.isend, send[me][1], up, self.group, tag=1),
               d.P2POp(d.isend, send[me][0], dn, self.group, tag=0),
               d.P2POp(d.irecv, recv[me][0], dn, self.group, tag=1),
               d.P2POp(d.irecv, recv[me][1], up, self.group, tag=0)]
        for r in d.batch_isend_irecv(ops):
            r.wait()


# ------------------------------------------------------------------ slabs

class LibpicSlab:
    """A libpic subdomain context in the form the stepper calls.  Device
    buffers are torch tensors and the transports move them on torch's
    current stream, so the context must run on that same stream: create it
    (torch_memory=True) while a non-default torch stream is current."""

    def __init__(self, ctx, migrant_capacity=0, id_base=0):
        import torch

        mem = getattr(ctx, "_mem", None)
        if mem is None or not mem.stream.cuda_stream or \
                mem.stream.cuda_stream != torch.cuda.current_stream().cuda_stream:
            raise ValueError("a slab context must run on the current, non-default torch stream "
                             "(create it with torch_memory=True inside torch.cuda.stream(...))")
        self.ctx = ctx
        ctx.set_subdomain(True, migrant_capacity, id_base)

    def step_stage(self, stage):
        self.ctx.step_stage(stage)

    def halo_floats(self, which, side):
        return self.ctx.halo_floats(which, side)

    def halo_pack(self, which, side, buf):
        self.ctx.halo_pack(which, side, buf.data_ptr())

    def halo_unpack(self, which, side, buf):
        self.ctx.halo_unpack(which, side, buf.data_ptr())

    def migrant_bytes(self):
        return self.ctx.migrant_bytes()

    def migrants_pack(self, side, buf):
        self.ctx.migrants_pack(side, buf.data_ptr())

    def migrants_accept(self, side, buf):
        self.ctx.migrants_accept(side, buf.data_ptr())


class SlabStepper:
    """Steps the slabs this process holds (ring positions ring.positions()),
    exchanging through `ring`.  new_buffer(kind, n) returns a zeroed buffer:
    kind "f" of n floats (field planes), "b" of n bytes (a migrant message)."""

    def __init__(self, slabs, ring, new_buffer):
        self.slabs = dict(zip(ring.positions(), slabs))
        self.ring = ring
        self.send, self.recv = {}, {}
        for key in FIELDS + (MIGRANTS,):
            self.send[key] = {}
            self.recv[key] = {}
            for p, s in self.slabs.items():
                if key == MIGRANTS:
                    nb = s.migrant_bytes()
                    self.send[key][p] = [new_buffer("b", nb), new_buffer("b", nb)]
                    self.recv[key][p] = [new_buffer("b", nb), new_buffer("b", nb)]
                else:
                    # message to side s; the one from side s is as long as
                    # the neighbour's to side 1 - s (same slab geometry)
                    self.send[key][p] = [new_buffer("f", s.halo_floats(key, side)) for side in (0, 1)]
                    self.recv[key][p] = [new_buffer("f", s.halo_floats(key, 1 - side)) for side in (0, 1)]

    def stage(self, stage):
        for s in self.slabs.values():
            s.step_stage(stage)

    def exchange(self, key):
        for p, s in self.slabs.items():
            for side in (0, 1):
                if key == MIGRANTS:
                    s.migrants_pack(side, self.send[key][p][side])
                else:
                    s.halo_pack(key, side, self.send[key][p][side])
        self.ring.swap(self.send[key], self.recv[key])
        for p, s in self.slabs.items():
            for side in (0, 1):
                if key == MIGRANTS:
                    s.migrants_accept(side, self.recv[key][p][side])
                else:
                    s.halo_unpack(key, side, self.recv[key][p][side])

    def prime(self):
        """Guard planes of E and B from the neighbours (after the fields
        were written, before the first step)."""
        self.exchange(pic.FIELD_E)
        self.exchange(pic.FIELD_B)

    def step(self, n=1, mark=None):
        """n steps; mark(label), when given, is called at the stage
        boundaries ("push", "exchange", "frames", "fields", "end") as they
        are enqueued (a timer records events there)."""
        mark = mark or (lambda label: None)
        for _ in range(n):
            mark("push")
            self.stage(pic.STAGE_PUSH)
            mark("exchange")
            self.exchange(pic.FIELD_J)
            self.exchange(MIGRANTS)
            mark("frames")
            self.stage(pic.STAGE_FRAMES)
            mark("fields")
            self.stage(pic.STAGE_B_FIRST)
            self.exchange(pic.FIELD_B)
            self.stage(pic.STAGE_E)
            self.exchange(pic.FIELD_E)
            self.stage(pic.STAGE_B_SECOND)
            self.exchange(pic.FIELD_B)
            mark("end")


def torch_buffers(device):
    """new_buffer for SlabStepper: zeroed torch tensors on `device`."""
    import torch

    def new_buffer(kind, n):
        return torch.zeros(int(n), dtype=torch.float32 if kind == "f" else torch.uint8, device=device)

    return new_buffer
