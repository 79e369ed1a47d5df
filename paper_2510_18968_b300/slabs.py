"""z-slab decomposition of one grid over several ranks (one GPU each).

The paper runs its grid as boxes per process with ghost zones synchronised
between them (Sec. III).  Here the boxes are z-slabs of the global grid and
the synchronisation is a deep halo exchanged once per step:

* rank r owns the z-layers [z0, z1) of the global grid (a balanced split)
  and its handle covers them plus H halo layers on every face that is not a
  boundary of the global domain (both faces when z is periodic; on a
  non-periodic grid a halo stops at the domain's face);
* H is the reach of one step: 3 cells per face-flux evaluation (the widest
  reconstruction stencil), times the face-flux evaluations of the scheme,
  plus one per Gauss's-law charge evaluation (halo_layers);
* the handle applies the outflow condition at its cut faces; the error that
  causes travels at most H layers per step and so never reaches an owned
  layer, and after every step each halo layer is overwritten with the
  owning rank's value of that layer.  Owned layers therefore evolve bit for
  bit as in one handle over the whole grid.

Each step's state (U, the primitives, the recovery guess) moves between
ranks as raw bytes (rmhd_get_state_layers / rmhd_set_state_layers), by
point-to-point sends (torch.distributed: NCCL on GPUs, gloo on CPUs) or, for
several handles in one process, by device copies (LocalExchange).  There is
no collective on the data path; diagnostics are summed with one all-reduce.

The plan (which layers a rank needs and from whom) is independent of what
steps the slabs: a `stepper` only has to provide layer_bytes(),
get_layers(k0, nk, out), set_layers(k0, nk, buf), step(dt) and new_buffer(n).
"""
from dataclasses import dataclass

import numpy as np

# face-flux evaluations per step of each IMEX scheme (rmhd.h RMHD_IMEX_*):
# Table imex forms F of both stages; SSP2(3,3,2) and SSP3(3,3,2) of all
# three; SSP3(4,3,3) of stages 2-4 (its first stage's F has weight 0)
FLUX_EVALUATIONS = {0: 2, 1: 3, 2: 3, 3: 3}
STENCIL_RADIUS = 3          # WENO5 faces read cells i-2 .. i+3 (TVD: 2)
QFLUX_GAUSS = 2


def halo_layers(params):
    """Layers one step can reach from a cell: 3 per face-flux evaluation, plus
    one per evaluation of the Gauss's-law charge (a central difference after
    every recovery whose primitives feed a flux, and after the last one)."""
    nflux = FLUX_EVALUATIONS[int(params.get("imex", 0))]
    h = STENCIL_RADIUS * nflux
    if int(params.get("qflux_mode", 0)) == QFLUX_GAUSS:
        h += nflux + 1
    return h


def split(nz, world):
    """Balanced contiguous split of nz layers: [(z0, z1)] per rank."""
    base, extra = divmod(nz, world)
    out, z = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


@dataclass
class Slab:
    rank: int
    world: int
    nz: int                 # global layers
    periodic: bool
    H: int
    z0: int                 # owned global range [z0, z1)
    z1: int
    lo: int                 # halo layers below / above the owned range
    hi: int

    @property
    def nz_local(self):
        return self.lo + (self.z1 - self.z0) + self.hi

    def global_layer(self, k):
        """Global layer of local layer k (wrapped when periodic)."""
        g = self.z0 - self.lo + k
        return g % self.nz if self.periodic else g

    def local_owned(self):
        """Local range of the owned layers."""
        return self.lo, self.lo + (self.z1 - self.z0)


def make_slab(nz, world, rank, H, periodic):
    z0, z1 = split(nz, world)[rank]
    if world == 1:
        return Slab(rank, world, nz, periodic, H, z0, z1, 0, 0)
    if z1 - z0 < 1:
        raise ValueError(f"rank {rank} owns no layer ({nz} layers over {world} ranks)")
    # H deep on a cut face; on a non-periodic grid it stops at the domain's
    # faces, where the handle's own boundary condition is the grid's
    lo = H if periodic else min(H, z0)
    hi = H if periodic else min(H, nz - z1)
    if periodic and lo + hi + (z1 - z0) > 3 * nz:
        raise ValueError("halo wider than the periodic grid")
    return Slab(rank, world, nz, periodic, H, z0, z1, lo, hi)


def exchange_plan(nz, world, H, periodic):
    """Per ordered pair (src, dst) of ranks, the transfers that fill dst's
    halo layers from src's owned ones: a list of (src local layer, dst local
    layer, count) runs; src == dst happens only with world == 1 (none)."""
    slabs = [make_slab(nz, world, r, H, periodic) for r in range(world)]
    owner = np.empty(nz, int)
    for s in slabs:
        owner[s.z0:s.z1] = s.rank
    plan = {}
    for d in slabs:
        lo_own, hi_own = d.local_owned()
        halo = [k for k in range(d.nz_local) if not (lo_own <= k < hi_own)]
        by_src = {}
        for k in halo:
            g = d.global_layer(k)
            src = slabs[owner[g]]
            by_src.setdefault(src.rank, []).append((g - src.z0 + src.lo, k))
        for r, pairs in by_src.items():
            pairs.sort()
            runs, cur = [], None
            for ks, kd in pairs:
                if cur and ks == cur[0] + cur[2] and kd == cur[1] + cur[2]:
                    cur[2] += 1
                else:
                    cur = [ks, kd, 1]
                    runs.append(cur)
            plan[(r, d.rank)] = [tuple(x) for x in runs]
    return slabs, plan


class DistExchange:
    """Halo exchange between ranks of a torch.distributed process group
    (NCCL with CUDA buffers, gloo with CPU buffers): after every step each
    rank sends its owned layers that others need and receives its halo, all
    point-to-point sends posted together."""

    def __init__(self, stepper, nz, H, periodic, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.slabs, self.plan = exchange_plan(nz, self.world, H, periodic)
        self.slab = self.slabs[self.rank]
        self.stepper = stepper
        lb = stepper.layer_bytes()
        self.send = {d: [(ks, n, stepper.new_buffer(n * lb)) for ks, kd, n in runs]
                     for (s, d), runs in self.plan.items() if s == self.rank and d != s}
        self.recv = {s: [(kd, n, stepper.new_buffer(n * lb)) for ks, kd, n in runs]
                     for (s, d), runs in self.plan.items() if d == self.rank and s != d}

    def exchange(self):
        dist = self.dist
        for runs in self.send.values():
            for k0, n, buf in runs:
                self.stepper.get_layers(k0, n, buf)
        ops = []
        for peer, runs in sorted(self.send.items()):
            for _, _, buf in runs:
                ops.append(dist.P2POp(dist.isend, buf, self._global(peer), self.group))
        for peer, runs in sorted(self.recv.items()):
            for _, _, buf in runs:
                ops.append(dist.P2POp(dist.irecv, buf, self._global(peer), self.group))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()
        for runs in self.recv.values():
            for k0, n, buf in runs:
                self.stepper.set_layers(k0, n, buf)

    def _global(self, r):
        return r if self.group is None else self.dist.get_global_rank(self.group, r)


class LocalExchange:
    """The same exchange between several steppers of one process (one GPU or
    the CPU): layers are packed from the source and unpacked into the
    destination directly, in the order DistExchange posts them."""

    def __init__(self, steppers, nz, H, periodic):
        self.steppers = steppers
        self.slabs, self.plan = exchange_plan(nz, len(steppers), H, periodic)

    def exchange(self):
        staged = []
        for (s, d), runs in sorted(self.plan.items()):
            if s == d:
                continue
            src = self.steppers[s]
            for ks, kd, n in runs:
                buf = src.new_buffer(n * src.layer_bytes())
                src.get_layers(ks, n, buf)
                staged.append((d, kd, n, buf))
        for d, kd, n, buf in staged:     # every send packed before any unpack
            self.steppers[d].set_layers(kd, n, buf)


def slab_arrays(slab, arr):
    """The slab's extended z-range of a global array (..., nz, ny, nx), with
    periodic wrap."""
    ks = [slab.global_layer(k) for k in range(slab.nz_local)]
    return np.ascontiguousarray(arr[..., ks, :, :])


class SolverStepper:
    """A library handle as a slab stepper (CUDA buffers, the handle's
    stream ordered with torch's current stream)."""

    def __init__(self, solver):
        self.s = solver

    def layer_bytes(self):
        return self.s.state_layer_bytes()

    def new_buffer(self, nbytes):
        import torch
        return torch.empty(nbytes, dtype=torch.uint8, device="cuda")

    def get_layers(self, k0, n, buf):
        self.s.get_state_layers(k0, n, buf)

    def set_layers(self, k0, n, buf):
        self.s.set_state_layers(k0, n, buf)

    def step(self, dt):
        self.s.step(dt, 1, sync=False)


def slab_params(params, slab):
    """Parameters of a slab's handle: its local layer count; the outflow
    condition at the cut faces (z periodic globally becomes outflow locally,
    the halo absorbing the difference)."""
    p = dict(params)
    n = list(p["n"])
    n[2] = slab.nz_local
    p["n"] = tuple(n)
    if slab.world > 1:
        bc = list(p["bc"])
        bc[2] = 1
        p["bc"] = tuple(bc)
    return p


def slab_solver(R, wl_params, prim, metric=None, sigma_profile=None, slab=None, stream=None):
    """A library handle for a slab of a global problem: its parameters, its
    extended range of the global metric (alpha, beta, gamma, K arrays of the
    global grid, or None for flat space), conductivity profile and initial
    primitives (global arrays, sliced here)."""
    s = R.Solver(slab_params(wl_params, slab), stream=stream)
    if metric is not None:
        s.set_metric(*[slab_arrays(slab, a) for a in metric])
    if sigma_profile is not None:
        s.set_sigma(slab_arrays(slab, sigma_profile))
    s.set_prims(slab_arrays(slab, prim))
    return s
