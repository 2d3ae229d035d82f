"""Row-split domain decomposition of one 2D problem over several ranks (one GPU each).

The grid's rows (y) are divided into contiguous slabs, one per rank.  A rank advances its
slab on the EXTENDED rows [j0 - H, j1 + H) with H = 4 halo rows on each side that touches
another rank: one two-stage step reaches two rows per stage (the y faces read cells j-1..j+2,
the x faces' tangential quartic rows j-2..j+2), so after a step the slab's own rows
[j0, j1) are exact while the outer halo rows are not.  Before the next step every rank
replaces its halo rows by the neighbours' freshly computed boundary rows (W, W_x, W_y of
H rows per side): ONE exchange per step, of 2 H rows x 12 values per column, instead of two
exchanges of 2 rows per stage; the cost is recomputing the 2 H halo rows.  Where a slab
touches the domain's own y boundary (transmissive or wall), it is not extended there and the
solver applies that boundary itself; a slab side that touches another rank uses the
transmissive boundary on its halo rows, whose effect never reaches the slab's own rows within
one step.  Periodic y: the slabs form a ring.

The exchange runs through torch.distributed (gloo on the CPU, NCCL between GPUs) as one
all_gather of every rank's two boundary blocks.  DecomposedRun takes any solver with
set_state(W, Wx, Wy), step(dt) and get_state() on host arrays [nvar][rows][nx] (the library's
gks.Solver, or, in the tests, the CPU reference) and moves the slab through host memory each
step; DeviceDecomposedRun keeps the slab resident on its GPU (a gks.Solver) and moves only
the boundary and halo rows, device to device (gks_get_rows_device / gks_set_rows_device and
a device all_gather).  Both build the slab's solver with a caller-supplied factory.
"""
from __future__ import annotations

import numpy as np

HALO = 4   # halo rows per side: the dependency radius (rows) of one two-stage step


def split_rows(ny: int, nranks: int) -> list[tuple[int, int]]:
    """Contiguous row ranges [j0, j1) of nearly equal size (the first ny % nranks slabs one row
    larger)."""
    if nranks < 1 or ny < nranks:
        raise ValueError("need 1 <= nranks <= ny")
    base, extra = divmod(ny, nranks)
    out, j = [], 0
    for r in range(nranks):
        n = base + (1 if r < extra else 0)
        out.append((j, j + n))
        j += n
    return out


class Slab:
    """Geometry of rank `rank`'s slab: its own rows [j0, j1), the extended rows the solver
    holds (global indices, taken modulo ny when the y direction is periodic), and the
    neighbours whose rows fill each halo."""

    def __init__(self, ny: int, rank: int, nranks: int, periodic_y: bool, halo: int = HALO):
        self.ny, self.rank, self.nranks, self.halo = ny, rank, nranks, halo
        self.periodic = periodic_y
        self.ranges = split_rows(ny, nranks)
        self.j0, self.j1 = self.ranges[rank]
        if nranks > 1 and min(j1 - j0 for j0, j1 in self.ranges) < halo:
            raise ValueError(f"every slab needs at least {halo} rows")
        if nranks == 1:
            self.lower = self.upper = None
        else:
            self.lower = (rank - 1) % nranks if (periodic_y or rank > 0) else None
            self.upper = (rank + 1) % nranks if (periodic_y or rank < nranks - 1) else None
        self.hl = halo if self.lower is not None else 0
        self.hu = halo if self.upper is not None else 0
        # global row of each extended row
        rows = np.arange(self.j0 - self.hl, self.j1 + self.hu)
        self.rows = rows % ny if periodic_y else rows
        self.n_ext = len(self.rows)

    @property
    def own(self) -> slice:
        """The slab's own rows within the extended arrays."""
        return slice(self.hl, self.hl + (self.j1 - self.j0))

    def local_bc_y(self, bc_y: int) -> int:
        """y boundary of the slab's solver: a periodic domain split over several ranks becomes
        transmissive (both slab ends carry halos); otherwise the domain's own boundary, which
        is right at the end that touches it and harmless beside a halo."""
        return 1 if (self.nranks > 1 and self.periodic) else bc_y

    def local_y_range(self, y0: float, y1: float) -> tuple[float, float]:
        """A y range of the extended rows whose cell size (y1' - y0')/n_ext equals the global
        dy = (y1 - y0)/ny to the last bit where such an extent exists (the scheme depends on dy,
        not on where the slab sits, so the range starts at 0); otherwise n_ext dy, whose cell
        size is within an ulp of dy (the slabs then differ from one domain by rounding)."""
        dy = (y1 - y0) / self.ny
        top = self.n_ext * dy
        up = down = top
        for _ in range(64):
            for cand in (up, down):
                if cand / self.n_ext == dy:
                    return 0.0, cand
            up = float(np.nextafter(up, np.inf))
            down = float(np.nextafter(down, -np.inf))
        return 0.0, top

    def extract(self, A: np.ndarray) -> np.ndarray:
        """The extended rows of a global array [nvar][ny][nx]."""
        return np.ascontiguousarray(A[:, self.rows, :])


def _boundary_blocks(slab: Slab, arrays) -> np.ndarray:
    """This rank's first and last `halo` own rows of every array: [2][narr][nvar][halo][nx]."""
    o = slab.own
    lo = np.stack([a[:, o.start:o.start + slab.halo, :] for a in arrays])
    hi = np.stack([a[:, o.stop - slab.halo:o.stop, :] for a in arrays])
    return np.stack([lo, hi])


def exchange_halos(slab: Slab, arrays, dist) -> None:
    """Overwrite the halo rows of `arrays` (W, Wx[, Wy], extended, in place) with the
    neighbours' boundary rows: the lower halo takes the lower neighbour's last rows, the
    upper halo the upper neighbour's first rows (one all_gather)."""
    if slab.nranks == 1:
        return
    import torch
    mine = torch.from_numpy(_boundary_blocks(slab, arrays))
    parts = [torch.empty_like(mine) for _ in range(slab.nranks)]
    dist.all_gather(parts, mine)
    h = slab.halo
    if slab.lower is not None:
        blk = parts[slab.lower][1].numpy()
        for a, b in zip(arrays, blk):
            a[:, :h, :] = b
    if slab.upper is not None:
        blk = parts[slab.upper][0].numpy()
        for a, b in zip(arrays, blk):
            a[:, a.shape[1] - h:, :] = b


class DecomposedRun:
    """One 2D problem advanced by `nranks` ranks, each holding one slab.

    make_solver(ny_ext, y0, y1, bc_y) builds the slab's solver for the extended rows (same nx,
    x domain, physics and scheme as the global problem).  W, Wx, Wy: the global initial state
    (every rank passes the same arrays)."""

    def __init__(self, W, Wx, Wy, y0: float, y1: float, bc_y: int, make_solver, rank: int,
                 nranks: int, dist=None, halo: int = HALO):
        self.nvar, ny, self.nx = W.shape
        self.slab = Slab(ny, rank, nranks, bc_y == 0, halo)
        self.dist = dist
        ly0, ly1 = self.slab.local_y_range(y0, y1)
        self.solver = make_solver(self.slab.n_ext, ly0, ly1, self.slab.local_bc_y(bc_y))
        self.state = [self.slab.extract(A) for A in (W, Wx, Wy)]
        self.solver.set_state(*self.state)

    def step(self, dt: float) -> None:
        """One two-stage step of the whole problem: the slab's step, then the halo exchange."""
        self.solver.step(dt)
        W, Wx, Wy = self.solver.get_state()
        self.state = [np.ascontiguousarray(W), np.ascontiguousarray(Wx), np.ascontiguousarray(Wy)]
        exchange_halos(self.slab, self.state, self.dist)
        self.solver.set_state(*self.state)

    def own_state(self):
        """This slab's own rows of W, Wx, Wy."""
        o = self.slab.own
        return [a[:, o, :].copy() for a in self.state]

    def gather(self):
        """The global state assembled on every rank (all_gather of the slabs, each padded to
        the largest slab's rows)."""
        return gather_slabs(self.slab, self.own_state(), self.dist)


def gather_slabs(slab: Slab, own, dist):
    """Assemble the global arrays from every rank's own rows (host arrays [nvar][rows][nx])."""
    if slab.nranks == 1:
        return own
    import torch
    sizes = [j1 - j0 for j0, j1 in slab.ranges]
    m = max(sizes)
    out = []
    for a in own:
        pad = torch.zeros((a.shape[0], m, a.shape[2]), dtype=torch.float64)
        pad[:, :a.shape[1], :] = torch.from_numpy(a)
        got = [torch.empty_like(pad) for _ in sizes]
        dist.all_gather(got, pad)
        out.append(torch.cat([g[:, :n, :] for g, n in zip(got, sizes)], dim=1).numpy())
    return out


class DeviceDecomposedRun:
    """One 2D problem advanced by `nranks` ranks with every slab resident on its GPU.

    make_solver(ny_ext, y0, y1, bc_y) builds the slab's gks.Solver (same nx, x domain,
    physics, scheme and precision as the global problem).  Per step: the slab's step; its
    first and last `halo` own rows of W, Wx, Wy packed on the device (gks_get_rows_device);
    one all_gather of the packed blocks (NCCL: device to device; another backend: staged
    through host memory); the neighbours' blocks written into the halo rows
    (gks_set_rows_device, which also refreshes the FP32-bulk form's float mirror of them).
    2 halo x 3 arrays x nvar x nx doubles per rank and step travel, nothing else."""

    def __init__(self, W, Wx, Wy, y0: float, y1: float, bc_y: int, make_solver, rank: int,
                 nranks: int, dist=None, halo: int = HALO, device=None):
        import torch
        self.nvar, ny, self.nx = W.shape
        self.slab = Slab(ny, rank, nranks, bc_y == 0, halo)
        self.dist = dist
        ly0, ly1 = self.slab.local_y_range(y0, y1)
        self.solver = make_solver(self.slab.n_ext, ly0, ly1, self.slab.local_bc_y(bc_y))
        self.solver.set_state(*[self.slab.extract(A) for A in (W, Wx, Wy)])
        self.device = torch.device("cuda") if device is None else torch.device(device)
        self.mine = torch.empty((2, 3, self.nvar, halo, self.nx), dtype=torch.float64,
                                device=self.device)
        self._staged = dist is not None and dist.get_backend() != "nccl"

    def pack(self):
        """This rank's boundary blocks [2][3][nvar][halo][nx] (device; synchronised)."""
        o, h = self.slab.own, self.slab.halo
        self.solver.get_rows_device(o.start, h, self.mine[0].data_ptr())
        self.solver.get_rows_device(o.stop - h, h, self.mine[1].data_ptr())
        self.solver.sync()
        return self.mine

    def unpack(self, parts):
        """Write the neighbours' boundary blocks (parts[r] = rank r's pack()) into the halo
        rows."""
        import torch
        h = self.slab.halo
        torch.cuda.current_stream(self.device).synchronize()
        if self.slab.lower is not None:
            blk = parts[self.slab.lower][1].to(self.device).contiguous()
            self.solver.set_rows_device(0, h, blk.data_ptr())
            self._keep = blk
        if self.slab.upper is not None:
            blk2 = parts[self.slab.upper][0].to(self.device).contiguous()
            self.solver.set_rows_device(self.slab.n_ext - h, h, blk2.data_ptr())
            self._keep2 = blk2
        self.solver.sync()

    def step(self, dt: float) -> None:
        """One two-stage step of the whole problem: the slab's step, then the halo exchange."""
        self.solver.step(dt)
        if self.slab.nranks == 1:
            return
        import torch
        mine = self.pack()
        if self._staged:
            mine = mine.cpu()
        parts = [torch.empty_like(mine) for _ in range(self.slab.nranks)]
        self.dist.all_gather(parts, mine)
        self.unpack(parts)

    def own_state(self):
        """This slab's own rows of W, Wx, Wy (host arrays)."""
        W, Wx, Wy = self.solver.get_state()
        o = self.slab.own
        return [a[:, o, :].copy() for a in (W, Wx, Wy)]

    def gather(self):
        return gather_slabs(self.slab, self.own_state(), self.dist)
