"""CPU check of the compressed grid's schedule (the ordering argument of the
GPU's one-buffer sweeps, Sect. 2.1 adapted to many concurrent work items).

The GPU pass reads the grid at one position of a buffer and writes the
result S = w*bz + D + 1 planes away, in items (x-y tile, z chunk) that take
tickets in chunk order (reversed on alternate passes) and wait for the items
of their own and the eight neighbouring tiles w and w+1 chunks back
(j -+ w, j -+ (w+1)).  This test restates the items' read and write sets
(the tile geometry of the register-blocked body: regions W x H with a margin
of D cells, pieces of A cells; the FP64 column walk: 32 x 8 columns with a
margin of one cell; the Dirichlet cells each item moves) and checks, for
many small configurations and both directions:

  * no item reads a cell it writes;
  * every cell of the grid at the write position is written by exactly one
    item;
  * whenever item I writes a cell that item V reads, V has a smaller ticket
    and V is among the items I waits for, directly or through the items
    those wait for (so V has finished before I starts, whatever the
    interleaving of the others).

A small simulation then runs the items in random orders that respect the
waits and the tickets (several in flight at once; an item reads its inputs
when it starts and again when it ends, and writes when it ends) and
compares the result with the oracle's sweeps.
"""

import numpy as np
import pytest

import oracle
from paper_1006_3148_gb300 import inputs


class Geometry:
    """Tiles of one pass: FP32 regions W x H (margin D, pieces of A cells),
    or the FP64 column tiles (32 x 8 by default, margin 1)."""

    def __init__(self, nx, ny, nz, D, bz, w, W=None, H=None, f64=False, tx=32, ty=8):
        self.nx, self.ny, self.nz, self.D, self.bz, self.w = nx, ny, nz, D, bz, w
        self.S = w * bz + D + 1
        if f64:
            assert D == 1
            self.bx, self.by, self.off, self.margin = tx, ty, 0, 1
            self.W = self.H = None
        else:
            A = 2 if (nx + 2) % 2 == 0 else 1
            self.off = ((1 - D) % A + A) % A
            self.bx = ((W - 2 * D - self.off) // A) * A
            self.by = H - 2 * D
            self.W, self.H = W, H
            assert self.bx > D and self.by > D
        self.f64 = f64
        self.ntx = -(-nx // self.bx)
        self.nty = -(-ny // self.by)
        self.nch = -(-nz // bz)
        self.shape = (nz + 2 + self.S, ny + 2, nx + 2)

    def z_range(self, j):
        z0 = 1 + j * self.bz
        return z0, min(z0 + self.bz, self.nz + 1)

    def footprint(self, tix, tiy):
        nx, ny = self.nx, self.ny
        fx0 = 0 if tix == 0 else 1 + tix * self.bx
        fx1 = nx + 2 if tix == self.ntx - 1 else 1 + (tix + 1) * self.bx
        fy0 = 0 if tiy == 0 else 1 + tiy * self.by
        fy1 = ny + 2 if tiy == self.nty - 1 else 1 + (tiy + 1) * self.by
        return fx0, fx1, fy0, fy1

    def item_sets(self, tix, tiy, j, up):
        """(read mask, write mask) over the buffer for item (tix, tiy, j)."""
        nx, ny, nz, D = self.nx, self.ny, self.nz, self.D
        src = self.S if up else 0
        dst = 0 if up else self.S
        rd = np.zeros(self.shape, bool)
        wr = np.zeros(self.shape, bool)
        z0, z1 = self.z_range(j)
        # body: region reads and tile writes
        if self.f64:
            xs0, xs1 = 1 + tix * self.bx, min(1 + (tix + 1) * self.bx, nx + 1)
            ys0, ys1 = 1 + tiy * self.by, min(1 + (tiy + 1) * self.by, ny + 1)
            # the column walk reads x-1..x+1, y-1..y+1 (no corners; a box is
            # a superset) and planes z0-1 .. z1
            rd[src + z0 - 1:src + z1 + 1, ys0 - 1:ys1 + 1, xs0 - 1:xs1 + 1] = True
        else:
            xa = 1 - D - self.off + tix * self.bx
            ya = 1 - D + tiy * self.by
            pz0 = max(0, z0 - D)
            pz1 = min(nz + 1, z1 - 1 + D)  # last plane loaded
            rd[src + pz0:src + pz1 + 1, max(ya, 0):min(ya + self.H, ny + 2), max(xa, 0):min(xa + self.W, nx + 2)] = True
            xs0, xs1 = 1 + tix * self.bx, min(1 + (tix + 1) * self.bx, nx + 1)
            ys0, ys1 = 1 + tiy * self.by, min(1 + (tiy + 1) * self.by, ny + 1)
        wr[dst + z0:dst + z1, ys0:ys1, xs0:xs1] = True
        # the Dirichlet cells of the footprint, moved from src to dst
        fx0, fx1, fy0, fy1 = self.footprint(tix, tiy)
        mv = np.zeros((nz + 2, ny + 2, nx + 2), bool)
        ring = np.zeros((ny + 2, nx + 2), bool)
        ring[0, :] = ring[ny + 1, :] = True
        ring[:, 0] = ring[:, nx + 1] = True
        fp = np.zeros((ny + 2, nx + 2), bool)
        fp[fy0:fy1, fx0:fx1] = True
        mv[z0:z1] |= (ring & fp)[None]
        if j == 0:
            mv[0] |= fp
        if j == self.nch - 1:
            mv[nz + 1] |= fp
        rd[src:src + nz + 2] |= mv
        wr[dst:dst + nz + 2] |= mv
        return rd, wr

    def items(self, up):
        """Items in ticket order: [(ticket, tix, tiy, j)]."""
        out = []
        ncols = self.ntx * self.nty
        for q in range(self.nch):
            j = q if up else self.nch - 1 - q
            for c in range(ncols):
                out.append((q * ncols + c, c % self.ntx, c // self.ntx, j))
        return out

    def waits(self, tix, tiy, j, up):
        """The items (tix', tiy', j') item (tix, tiy, j) waits for."""
        out = set()
        for l in range(18):
            nx_, ny_ = tix + l % 3 - 1, tiy + (l // 3) % 3 - 1
            jj = j - self.w - l // 9 if up else j + self.w + l // 9
            if 0 <= nx_ < self.ntx and 0 <= ny_ < self.nty and 0 <= jj < self.nch:
                out.add((nx_, ny_, jj))
        return out


def _check_static(g, up):
    its = g.items(up)
    key = {(tx, ty, j): t for t, tx, ty, j in its}
    sets = {(tx, ty, j): g.item_sets(tx, ty, j, up) for _, tx, ty, j in its}
    # transitive closure of the waits (items with smaller tickets only)
    closure = {}
    for t, tx, ty, j in its:  # ticket order: waits are already closed
        c = set()
        for d in g.waits(tx, ty, j, up):
            assert key[d] < t, "wait on a later ticket"
            c.add(d)
            c |= closure[d]
        closure[(tx, ty, j)] = c
    cover = np.zeros(g.shape, np.int32)
    for k, (rd, wr) in sets.items():
        assert not (rd & wr).any(), ("item reads what it writes", k)
        cover += wr
    dst = 0 if up else g.S
    assert (cover[dst:dst + g.nz + 2] == 1).all(), "grid not written exactly once"
    assert cover.sum() == (g.nz + 2) * (g.ny + 2) * (g.nx + 2)
    for ki, (_, wi) in sets.items():
        for kv, (rv, _) in sets.items():
            if ki == kv:
                continue
            if (wi & rv).any():
                assert kv in closure[ki], ("item %s overwrites input of %s, which it does not wait for" % (ki, kv))


CONFIGS = [
    # nx, ny, nz, D, bz, w, W, H
    (14, 11, 24, 1, 4, 1, 8, 6),
    (15, 9, 30, 2, 6, 1, 10, 8),
    (16, 12, 40, 3, 8, 1, 12, 10),
    (13, 13, 40, 3, 8, 2, 12, 10),
    (18, 10, 45, 4, 10, 1, 16, 14),
    (17, 14, 37, 2, 7, 2, 10, 9),
    (12, 20, 50, 3, 9, 3, 12, 10),
    (20, 7, 50, 1, 4, 2, 8, 5),
]


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: "x".join(map(str, c)))
def test_fp32_items_never_overwrite_unread_input(cfg):
    nx, ny, nz, D, bz, w, W, H = cfg
    g = Geometry(nx, ny, nz, D, bz, w, W, H)
    assert g.ntx >= 2 and g.nty >= 2 and g.nch >= w + 2
    for up in (1, 0):
        _check_static(g, up)


@pytest.mark.parametrize("cfg", [(40, 20, 30, 4, 1), (70, 17, 26, 5, 2), (33, 9, 40, 4, 3)])
def test_fp64_items_never_overwrite_unread_input(cfg):
    nx, ny, nz, bz, w = cfg
    g = Geometry(nx, ny, nz, 1, bz, w, f64=True, tx=16, ty=4)
    for up in (1, 0):
        _check_static(g, up)


@pytest.mark.parametrize("cfg", [(16, 12, 40, 3, 1, 8, 1, 12, 10), (18, 10, 45, 4, 2, 10, 1, 14, 12),
                                 (17, 14, 37, 2, 1, 7, 2, 10, 9)])
def test_shallower_last_pass_keeps_the_deeper_shift(cfg):
    # a last pass of depth d < D runs its own tiles but the shift of depth D
    nx, ny, nz, D, d, bz, w, W, H = cfg
    g = Geometry(nx, ny, nz, d, bz, w, W, H)
    g.S = w * bz + D + 1
    g.shape = (g.nz + 2 + g.S, g.ny + 2, g.nx + 2)
    for up in (1, 0):
        _check_static(g, up)


def test_a_shift_one_plane_short_is_caught():
    # the same geometry with S one plane smaller must fail the check
    g = Geometry(16, 12, 40, 3, 8, 1, 12, 10)
    g.S -= 1
    g.shape = (g.nz + 2 + g.S, g.ny + 2, g.nx + 2)
    with pytest.raises(AssertionError):
        _check_static(g, 1)


def test_waiting_on_one_chunk_only_is_caught():
    # with w >= 2 the items w+1 chunks back are not among those the w-back
    # items wait for, so dropping that wait must fail (with w = 1 it is
    # implied: the items one chunk back waited for those two back)
    g = Geometry(13, 13, 40, 3, 8, 2, 12, 10)
    full = g.waits
    g.waits = lambda tx, ty, j, up: {d for d in full(tx, ty, j, up) if abs(d[2] - j) == g.w}
    with pytest.raises(AssertionError):
        _check_static(g, 1)


# ------------------------------------------------------------ value simulation

def _jacobi_block(block, fixed, levels):
    """levels sweeps of Eq. (1) on a block; cells with fixed=True keep their
    values (the Dirichlet cells and the block's outer layer)."""
    cur = block.copy()
    for _ in range(levels):
        new = cur.copy()
        s = cur[1:-1, 1:-1, :-2] + cur[1:-1, 1:-1, 2:]
        s = s + cur[1:-1, :-2, 1:-1]
        s = s + cur[1:-1, 2:, 1:-1]
        s = s + cur[:-2, 1:-1, 1:-1]
        s = s + cur[2:, 1:-1, 1:-1]
        # the order above regroups Eq. (1)'s sum: the simulation compares
        # within a tolerance, not bitwise
        upd = s / 6.0
        inner = new[1:-1, 1:-1, 1:-1]
        keep = fixed[1:-1, 1:-1, 1:-1]
        inner[~keep] = upd[~keep]
        cur = new
    return cur


def _simulate(g, a, T, rng, inflight=4):
    nz2, ny2, nx2 = a.shape
    U = np.full(g.shape, np.nan)
    U[g.S:g.S + nz2] = a
    up = 1
    halo = np.ones(a.shape, bool)
    halo[1:-1, 1:-1, 1:-1] = False
    P = -(-T // g.D)
    for p in range(P):
        d = min(g.D, T - p * g.D)
        src = g.S if up else 0
        dst = 0 if up else g.S
        its = g.items(up)
        done, running, nxt = set(), [], 0
        snap = {}
        while nxt < len(its) or running:
            can_start = nxt < len(its) and len(running) < inflight and all(
                w_ in done for w_ in g.waits(*its[nxt][1:], up))
            if can_start and (not running or rng.random() < 0.5):
                _, tx, ty, j = its[nxt]
                rd, _ = g.item_sets(tx, ty, j, up)
                snap[(tx, ty, j)] = U[rd].copy()
                running.append((tx, ty, j))
                nxt += 1
                continue
            k = running.pop(int(rng.integers(0, len(running))))
            rd, wr = g.item_sets(*k, up)
            assert np.array_equal(U[rd], snap.pop(k), equal_nan=True), ("input changed while in flight", k)
            # result of this item from the logical grid at the src position
            grid = U[src:src + nz2]
            fixed = halo.copy()
            res = _jacobi_block(grid, fixed, d)
            sel = wr[dst:dst + nz2]
            # Dirichlet cells are copied, interior cells take the swept values
            vals = np.where(halo, grid, res)
            U[dst:dst + nz2][sel] = vals[sel]
            done.add(k)
        up = 1 - up
    return U[(g.S if up else 0):(g.S if up else 0) + nz2]


@pytest.mark.parametrize("cfg,T", [((14, 11, 24, 1, 4, 1, 8, 6), 3), ((16, 12, 40, 3, 8, 1, 12, 10), 7),
                                   ((13, 13, 40, 3, 8, 2, 12, 10), 5)])
def test_random_schedules_reach_the_oracle(cfg, T):
    nx, ny, nz, D, bz, w, W, H = cfg
    g = Geometry(nx, ny, nz, D, bz, w, W, H)
    a = inputs.uniform_grid(nx, ny, nz, seed=3).numpy()
    exp = oracle.jacobi_result(a, T)
    for seed in range(3):
        got = _simulate(g, a, T, np.random.default_rng(seed))
        assert not np.isnan(got).any()
        assert np.abs(got - exp).max() <= 1e-13
