"""Models of the two Gauss-Seidel schedules that run without grid barriers,
executed on the CPU under random interleavings of the blocks.

* 7-point (hs_gs.cu): tiles are a dataflow graph.  Blocks claim (sweep, tile)
  items from a counter in step order (sweep t's tile plane S at step
  off(t) + S, off(t) = 2t for one direction, t P for alternating symmetric
  sweeps); before sweeping a tile a block waits until the tile and its
  old-side face neighbours have completed the previous sweep and its
  new-side face neighbours the current one.
* 27-point (hs_gs27.cu): one step per point hyperplane i + 2j + 4k, z planes
  dealt to blocks round robin, sweeps of one direction pipelined 8
  hyperplanes apart; before a step with work a block waits until both ring
  neighbours have completed the previous step.

Each block step is modelled as a read phase and a later write phase with
other blocks' events in between, so a missing wait shows up as a value read
in the wrong state.  The result must equal the sequential sweep, and the
models must fail when a wait the kernels rely on is dropped (the test would
otherwise prove nothing).  Small grids; plain Python."""
import itertools
import random

import numpy as np
import pytest


def _seq_sweeps(x, b, nbrs, order, dirs, diag):
    x = x.copy()
    for bw in dirs:
        for p in (reversed(order) if bw else order):
            x[p] = (b[p] + sum(x[q] for q in nbrs(p))) / diag
    return x


# ---------------------------------------------------------------- 7-point

def _model_gs7(shape, tiles, G, dirs, seed, drop_old_side=False):
    nx, ny, nz = shape
    TX, TY, TZ = tiles
    ntx, nty, ntz = -(-nx // TX), -(-ny // TY), -(-nz // TZ)
    nt = ntx * nty * ntz
    P = ntx + nty + ntz - 2
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (nx, ny, nz))
    b = rng.uniform(-1, 1, (nx, ny, nz))

    def nbrs(p):
        i, j, k = p
        for d in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            q = (i + d[0], j + d[1], k + d[2])
            if 0 <= q[0] < nx and 0 <= q[1] < ny and 0 <= q[2] < nz:
                yield q

    order = [(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)]
    ref = _seq_sweeps(x, b, nbrs, order, dirs, 6.5)
    planes = {}
    for t in range(nt):
        planes.setdefault(t % ntx + (t // ntx) % nty + t // (ntx * nty), []).append(t)
    L = P if len(set(dirs)) > 1 else 2
    seq, tau = [], 0
    while len(seq) < len(dirs) * nt:
        for s in range(len(dirs)):
            S = tau - L * s
            if 0 <= S < P:
                for tl in planes.get(P - 1 - S if dirs[s] else S, []):
                    seq.append((s, tl))
        tau += 1

    def deps(u):
        s, tile = seq[u]
        I, J, K = tile % ntx, (tile // ntx) % nty, tile // (ntx * nty)
        out = [(tile, s)]
        for c, lim, stp in ((I, ntx, 1), (J, nty, ntx), (K, ntz, ntx * nty)):
            for up in (0, 1):
                cc = c + (1 if up else -1)
                if 0 <= cc < lim:
                    newside = up if dirs[s] else not up
                    if newside:
                        out.append((tile + (stp if up else -stp), s + 1))
                    elif not drop_old_side:
                        out.append((tile + (stp if up else -stp), s))
        return out

    done = [0] * nt
    claim, state, finished = 0, [None] * G, [False] * G
    rnd = random.Random(seed)
    while not all(finished):
        g = rnd.randrange(G)
        if finished[g]:
            continue
        st = state[g]
        if st is None:
            if claim >= len(seq):
                finished[g] = True
                continue
            state[g] = ("wait", claim)
            claim += 1
        elif st[0] == "wait":
            u = st[1]
            if all(done[t] >= n for t, n in deps(u)):
                s, tile = seq[u]
                I, J, K = tile % ntx, (tile // ntx) % nty, tile // (ntx * nty)
                loc = x.copy()   # the tile and its halo as staged
                pts = [(i, j, k) for k in range(K * TZ, min(nz, K * TZ + TZ))
                       for j in range(J * TY, min(ny, J * TY + TY)) for i in range(I * TX, min(nx, I * TX + TX))]
                for p in (reversed(pts) if dirs[s] else pts):
                    loc[p] = (b[p] + sum(loc[q] for q in nbrs(p))) / 6.5
                state[g] = ("staged", u, {p: loc[p] for p in pts})
        else:
            for p, v in st[2].items():
                x[p] = v
            s, tile = seq[st[1]]
            done[tile] = s + 1
            state[g] = None
    return np.max(np.abs(x - ref))


@pytest.mark.parametrize("shape,tiles", [((7, 5, 6), (3, 2, 2)), ((9, 2, 3), (4, 1, 1)), ((5, 5, 1), (2, 2, 1))])
@pytest.mark.parametrize("G", [1, 3, 6])
@pytest.mark.parametrize("dirs", [(False,), (False, False, False), (True, True), (False, True, False, True)])
def test_gs7_dataflow_schedule_equals_sequential_sweeps(shape, tiles, G, dirs):
    assert _model_gs7(shape, tiles, G, list(dirs), seed=hash((shape, G, dirs)) % 9973) < 1e-12


def test_gs7_model_detects_a_dropped_old_side_wait():
    errs = [_model_gs7((4, 4, 4), (2, 2, 2), 6, [False] * 3, seed=s, drop_old_side=True) for s in range(6)]
    assert max(errs) > 1e-6


# --------------------------------------------------------------- 27-point

def _model_gs27(shape, G, batches, seed, drop_upper_wait=False):
    nx, ny, nz = shape
    H = (nx - 1) + 2 * (ny - 1) + 4 * (nz - 1) + 1
    M = nx // 2 + 1
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (nx, ny, nz))
    b = rng.uniform(-1, 1, (nx, ny, nz))

    def nbrs(p):
        i, j, k = p
        for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
            q = (i + dx, j + dy, k + dz)
            if q != p and 0 <= q[0] < nx and 0 <= q[1] < ny and 0 <= q[2] < nz:
                yield q

    order = [(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)]
    dirs = [bw for nsw, bw in batches for _ in range(nsw)]
    ref = _seq_sweeps(x, b, nbrs, order, dirs, 27.0)

    def plane_nodes(h, bblk):
        khi = min(nz - 1, h // 4)
        r = h - (nx - 1) - 2 * (ny - 1)
        klo = 0 if r <= 0 else (r + 3) // 4
        out = []
        if klo > khi:
            return out
        k0 = klo + ((bblk - klo % G) % G + G) % G
        cnt = (khi - k0) // G + 1 if k0 <= khi else 0
        for loc in range(cnt * M):
            k = k0 + (loc // M) * G
            rem = h - 4 * k
            jlo = 0 if rem - (nx - 1) <= 0 else (rem - (nx - 1) + 1) // 2
            j = jlo + loc % M
            if j < ny and 2 * j <= rem:
                out.append((rem - 2 * j, j, k))
        return out

    sched = [(nsw, bw, tau) for nsw, bw in batches for tau in range(H + 8 * (nsw - 1))]
    prog, pos, pending, fin = [0] * G, [0] * G, [None] * G, [False] * G
    rnd = random.Random(seed)
    while not all(fin):
        g = rnd.randrange(G)
        if fin[g]:
            continue
        if pos[g] >= len(sched):
            fin[g] = True
            continue
        nsw, bw, tau = sched[pos[g]]
        if pending[g] is None:
            nodes = []
            for t in range(min(nsw - 1, tau // 8), -1, -1):
                s = tau - 8 * t
                if s >= H:
                    break
                nodes += plane_nodes(H - 1 - s if bw else s, g)
            if not nodes:
                pos[g] += 1
                prog[g] = pos[g]
                continue
            if prog[(g - 1) % G] < pos[g] or (not drop_upper_wait and prog[(g + 1) % G] < pos[g]):
                continue
            pending[g] = [(p, (b[p] + sum(x[q] for q in nbrs(p))) / 27.0) for p in nodes]
        else:
            for p, v in pending[g]:
                x[p] = v
            pending[g] = None
            pos[g] += 1
            prog[g] = pos[g]
    return np.max(np.abs(x - ref))


@pytest.mark.parametrize("shape", [(5, 4, 3), (1, 9, 7), (8, 1, 5), (3, 2, 20)])
@pytest.mark.parametrize("G", [1, 2, 5])
@pytest.mark.parametrize("batches", [((1, False),), ((3, False),), ((1, False), (1, True), (1, False)),
                                     ((4, True), (2, False))])
def test_gs27_ring_schedule_equals_sequential_sweeps(shape, G, batches):
    assert _model_gs27(shape, G, list(batches), seed=hash((shape, G, batches)) % 9973) < 1e-12


def test_gs27_model_detects_a_dropped_upper_wait():
    errs = [_model_gs27((9, 3, 11), 5, [(3, False)], seed=s, drop_upper_wait=True) for s in range(4)]
    assert max(errs) > 1e-6


# ---------------------------------------------------------------------------
# Single-block shared-memory Gauss-Seidel for small 2-D grids (k_gs2d): sweep
# t works on anti-diagonal s - 2t at step s; thread (i, q) owns column i and
# the sweeps t = q (mod Q).  The model transcribes the kernel's index
# arithmetic and checks coverage and the order of every dependency.
# ---------------------------------------------------------------------------

def gs2d_schedule(nx, ny, nsw, threads, bw):
    Q = threads // nx
    dmax = nx + ny - 2
    visit = {}
    for s in range(dmax + 1 + 2 * (nsw - 1)):
        for tid in range(threads):
            i, q = tid % nx, tid // nx
            if q >= Q:
                continue
            t_lo = max(0, (s - i - (ny - 1) + 1) >> 1)
            t_hi = min(nsw - 1, (s - i) >> 1)
            t = t_lo + (((q - t_lo) % Q) + Q) % Q
            while t <= t_hi:
                r = s - 2 * t - i
                assert 0 <= r < ny
                node = (t, nx - 1 - i if bw else i, ny - 1 - r if bw else r)
                assert node not in visit, "node visited twice"
                visit[node] = s
                t += Q
    return visit


@pytest.mark.parametrize("nx,ny,nsw,threads", [(5, 4, 3, 20), (7, 1, 5, 21), (1, 1, 4, 32), (3, 9, 6, 30),
                                               (70, 45, 4, 980), (33, 1, 7, 1023), (1, 5, 3, 1024),
                                               (40, 30, 9, 1000)])
@pytest.mark.parametrize("bw", [False, True])
def test_gs2d_wavefront_schedule(nx, ny, nsw, threads, bw):
    visit = gs2d_schedule(nx, ny, nsw, threads, bw)
    assert len(visit) == nsw * nx * ny
    for (t, i, j), s in visit.items():
        new_side = [(i - 1, j), (i, j - 1)] if not bw else [(i + 1, j), (i, j + 1)]
        old_side = [(i + 1, j), (i, j + 1)] if not bw else [(i - 1, j), (i, j - 1)]
        for a, b in new_side:
            if 0 <= a < nx and 0 <= b < ny:
                assert visit[(t, a, b)] < s          # already updated in this sweep
        for a, b in old_side:
            if 0 <= a < nx and 0 <= b < ny:
                assert visit[(t, a, b)] > s          # not yet overwritten by this sweep
                if t > 0:
                    assert visit[(t - 1, a, b)] < s  # the previous sweep's value is there
        if t > 0:
            assert visit[(t - 1, i, j)] < s


def test_gs2d_schedule_model_catches_one_diagonal_shift():
    # sweeps one diagonal apart instead of two: a node reads a neighbour that
    # a later sweep updates in the same step
    nx, ny, nsw = 6, 5, 3
    visit = {}
    for s in range(nx + ny - 1 + (nsw - 1)):
        for t in range(nsw):
            for i in range(nx):
                r = s - t - i
                if 0 <= r < ny:
                    visit[(t, i, r)] = s
    with pytest.raises(AssertionError):
        for (t, i, j), s in visit.items():
            for a, b in [(i + 1, j), (i, j + 1)]:
                if a < nx and b < ny and t > 0:
                    assert visit[(t - 1, a, b)] < s
