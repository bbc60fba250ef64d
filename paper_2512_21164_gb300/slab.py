"""Slab partitioning of one stencil system over several ranks (one GPU each):
the plan, the halo exchange and the partitioned operator application.

One system of the 2D or 3D stencil classes is cut along its slowest axis (y in
2D, z in 3D) into contiguous slabs of whole planes, one per rank, balanced to
within one plane.  Every matrix-vector product of Algorithm 1 (A x for the
residual, H p in CG on alpha I + M, S p and S^T u in CGNR on alpha I + N)
couples a plane only with the planes next to it, so a rank needs

  * one ghost plane from each neighbour before an operator application (A,
    M, N, H, S or S^T), and
  * two ghost planes before the fused S^T (S p) of CGNR (S p is formed on the
    slab plus one plane on each side, then S^T on the slab),

and every dot product (p.Hp, r.r, u.u, t.t, ||b - A x||^2) is a local partial
sum followed by one all-reduce of the partials (two scalars per CG or CGNR
iteration, one per outer residual norm).  The planes at the ends of the grid
have zero ghosts (the Dirichlet boundary).

The local operator application is given as a callable on a slab grid
extended by its ghost planes, so the same code drives the CUDA library
(`gadi_apply` on a handle of the extended sub-grid, with the full grid's h)
and any other implementation of the same stencil.  Applying the stencil to
the extended grid and keeping the slab's planes gives, plane for plane, the
operations and operation order of the undivided grid, so the partitioned
product equals the single-rank product bit for bit.

Transport is torch.distributed point-to-point (NCCL between GPUs, gloo on
CPU); ghost planes travel as contiguous tensors, no remote-memory access or
multicast is used.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class SlabPlan:
    """Planes [lo, hi) of a grid with `planes` planes of `plane_elems`
    elements each, owned by `rank` of `world`."""

    planes: int
    plane_elems: int
    world: int
    rank: int
    lo: int
    hi: int

    @property
    def own(self) -> int:
        return self.hi - self.lo

    @property
    def prev(self) -> int | None:
        """Rank holding the planes below lo (None at the grid's edge)."""
        return self.rank - 1 if self.rank > 0 else None

    @property
    def next(self) -> int | None:
        return self.rank + 1 if self.rank + 1 < self.world else None

    def local_len(self, depth: int = 0) -> int:
        """Elements of the slab extended by `depth` ghost planes on each side."""
        return (self.own + 2 * depth) * self.plane_elems


def make_plan(planes: int, plane_elems: int, world: int, rank: int) -> SlabPlan:
    """Balanced contiguous split: rank r owns planes [r P / W, (r+1) P / W)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world / rank")
    if planes < world:
        raise ValueError(f"{planes} planes cannot be split over {world} ranks")
    lo = rank * planes // world
    hi = (rank + 1) * planes // world
    return SlabPlan(planes, plane_elems, world, rank, lo, hi)


def plan_for_grid(kind: int, nx: int, ny: int, nz: int, world: int, rank: int, complex_pairs: bool = False):
    """Plan for a stencil grid: 2D (kind 0, or 2 for the complex class) split
    along y, 3D (kind 1) along z; complex points carry two doubles."""
    per_pt = 2 if (complex_pairs or kind == 2) else 1
    if kind == 1:
        return make_plan(nz, nx * ny * per_pt, world, rank)
    return make_plan(ny, nx * per_pt, world, rank)


def extend(plan: SlabPlan, x_own, depth: int, group=None):
    """The slab vector extended by `depth` ghost planes on each side, filled
    from the neighbours (zeros at the grid's edges).  x_own: 1-D tensor of
    plan.local_len(0) elements.  Every rank sends its first and last `depth`
    planes and receives the neighbours' in one exchange."""
    import torch
    import torch.distributed as dist
    pe = plan.plane_elems
    if depth > plan.own:
        raise ValueError("halo deeper than the slab")
    ext = torch.zeros(plan.local_len(depth), dtype=x_own.dtype, device=x_own.device)
    ext[depth * pe: depth * pe + x_own.numel()] = x_own
    if plan.world == 1 or depth == 0:
        return ext
    ops, recv = [], []
    if plan.prev is not None:
        ops.append(dist.P2POp(dist.isend, x_own[:depth * pe].contiguous(), plan.prev, group))
        buf = torch.empty(depth * pe, dtype=x_own.dtype, device=x_own.device)
        ops.append(dist.P2POp(dist.irecv, buf, plan.prev, group))
        recv.append((0, buf))
    if plan.next is not None:
        ops.append(dist.P2POp(dist.isend, x_own[-depth * pe:].contiguous(), plan.next, group))
        buf = torch.empty(depth * pe, dtype=x_own.dtype, device=x_own.device)
        ops.append(dist.P2POp(dist.irecv, buf, plan.next, group))
        recv.append((ext.numel() - depth * pe, buf))
    for w in dist.batch_isend_irecv(ops):
        w.wait()
    for off, buf in recv:
        ext[off:off + buf.numel()] = buf
    return ext


def extend_from_full(plan: SlabPlan, x_full, depth: int):
    """What `extend` delivers, taken from a full-grid vector held by one
    process (zeros beyond the grid's edges): for running the ranks of a plan
    one after another in a single process."""
    import torch
    pe = plan.plane_elems
    ext = torch.zeros(plan.local_len(depth), dtype=x_full.dtype, device=x_full.device)
    a = max(plan.lo - depth, 0)
    b = min(plan.hi + depth, plan.planes)
    off = (a - (plan.lo - depth)) * pe
    ext[off: off + (b - a) * pe] = x_full[a * pe: b * pe]
    return ext


def interior(plan: SlabPlan, v_ext, depth: int):
    """The slab's own planes of an extended vector."""
    pe = plan.plane_elems
    return v_ext[depth * pe: depth * pe + plan.local_len(0)]


def apply_partitioned(plan: SlabPlan, apply_ext, x_own, group=None, x_ext=None):
    """y_own = (Op x)_slab for a nearest-plane stencil Op: one ghost plane per
    side, `apply_ext(x_ext, planes)` applies Op on the extended slab grid of
    `planes` planes (zero outside it) and returns a vector of the same
    length; the ghost planes' results are dropped.  x_ext (optional): the
    extended vector already at hand (then no exchange)."""
    if x_ext is None:
        x_ext = extend(plan, x_own, 1, group)
    y_ext = apply_ext(x_ext, plan.own + 2)
    return interior(plan, y_ext, 1)


def apply_normal_partitioned(plan: SlabPlan, apply_s_ext, apply_st_ext, p_own, group=None, p_ext=None):
    """(S^T (S p))_slab with two ghost planes per side (CGNR's fused product):
    u = S p on the slab plus one plane each side, then S^T u on the slab.
    Returns (w_own, u_own) -- u_own = (S p)_slab, whose squared norm CGNR
    needs.  p_ext (optional): p with its two ghost planes already at hand."""
    if p_ext is None:
        p_ext = extend(plan, p_own, 2, group)
    u2 = apply_s_ext(p_ext, plan.own + 4)
    pe = plan.plane_elems
    u1 = u2[pe: pe + plan.local_len(1)]
    # u on a plane outside the grid does not exist (zero Dirichlet value),
    # although S p evaluated there would not vanish: clear it at the edges.
    # (The outermost planes of u2 saw zeros beyond p's two ghost planes; they
    # are not part of u1.)
    u1 = u1.clone()
    if plan.prev is None:
        u1[:pe] = 0
    if plan.next is None:
        u1[-pe:] = 0
    w1 = apply_st_ext(u1, plan.own + 2)
    return interior(plan, w1, 1), interior(plan, u1, 1)


def allreduce_sum(values, group=None, device=None):
    """Sum per-rank partials (a list of floats) over the ranks in one
    all-reduce; returns a list of floats.  Every rank gets the same totals."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return [float(v) for v in t.tolist()]


class LibraryStencil:
    """The local operator products of a slab through the CUDA library:
    `gadi_apply` on handles of the extended sub-grids (the same stencil
    and the full grid's h, one handle per plane count, created on first
    use).  `op(which)` gives the callable `apply_partitioned` takes; vectors
    are FP64 device tensors."""

    def __init__(self, kind, nx, ny, nz, h, beta, kappa=0.0, sigma=0.0):
        self.kind, self.nx, self.ny, self.nz = kind, nx, ny, nz
        self.h, self.beta, self.kappa, self.sigma = h, tuple(beta), kappa, sigma
        self._handles = {}

    def _handle(self, planes):
        from . import Gadi, STENCIL_3D7
        if planes not in self._handles:
            if self.kind == STENCIL_3D7:
                dims = (self.nx, self.ny, planes)
            else:
                dims = (self.nx, planes, 1)
            self._handles[planes] = Gadi(self.kind, *dims, h=self.h, beta=self.beta, kappa=self.kappa,
                                         sigma=self.sigma)
        return self._handles[planes]

    def op(self, which):
        def apply(v_ext, planes):
            import torch
            y = torch.empty_like(v_ext)
            self._handle(planes).apply(which, v_ext, y)
            return y
        return apply

    def close(self):
        for h in self._handles.values():
            h.close()
        self._handles.clear()
