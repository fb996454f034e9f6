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
  neighbours have completed the previous step.  And the plane-lagged form
  (k_gs27p): whole planes per block, in-plane steps i + 2j, each plane four
  steps behind the one below it in the sweep and one sweep behind the one
  above.

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


def _model_gs27p(shape, G, dirs, seed, PUB=2, lag=4, drop_old_side=False):
    """The plane-lagged 27-point schedule (hs_gs27.cu, k_gs27p).  Block g owns
    planes k = g (mod G) and takes its items (t, k) sweep by sweep, planes in
    the sweep's direction.  An item first waits until the old-side plane (k+1
    forward, k-1 backward) has finished sweep t-1 (count >= t R), stages plane
    k (a private copy, like shared memory), then runs the rem steps
    r = i + 2j (sweep frame) in order: before step r it publishes its count
    t R + r when r % PUB == 0 and waits until the new-side plane's count is
    >= t R + min(r + lag, R); a step reads, then (after other blocks' events)
    writes both the copy and the global iterate.  A finished plane publishes
    (t + 1) R."""
    nx, ny, nz = shape
    R = (nx - 1) + 2 * (ny - 1) + 1
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
    ref = _seq_sweeps(x, b, nbrs, order, dirs, 27.0)
    G = min(G, nz)
    prog = [0] * nz

    def items(g):
        for t, bw in enumerate(dirs):
            ks = list(range(g, nz, G))
            for k in (reversed(ks) if bw else ks):
                yield t, k, bw

    def block(g):
        # a generator: yields whenever it has to wait or between a step's
        # read and write phases, so that other blocks interleave
        for t, k, bw in items(g):
            kp, kn = (k + 1, k - 1) if bw else (k - 1, k + 1)
            if 0 <= kn < nz and not drop_old_side:
                while prog[kn] < t * R:
                    yield
            xs = x[:, :, k].copy()
            for r in range(R):
                if r > 0 and r % PUB == 0:
                    prog[k] = t * R + r
                if 0 <= kp < nz:
                    while prog[kp] < t * R + min(r + lag, R):
                        yield
                nodes = []
                for j in range(max(0, -(-(r - nx + 1) // 2)), min(ny - 1, r // 2) + 1):
                    i = r - 2 * j
                    nodes.append((nx - 1 - i, ny - 1 - j) if bw else (i, j))
                new = []
                for i, j in nodes:
                    acc = b[i, j, k]
                    for q in nbrs((i, j, k)):
                        acc += xs[q[0], q[1]] if q[2] == k else x[q]
                    new.append(acc / 27.0)
                yield
                for (i, j), v in zip(nodes, new):
                    xs[i, j] = v
                    x[i, j, k] = v
            prog[k] = (t + 1) * R

    gens = [block(g) for g in range(G)]
    live = list(range(G))
    rnd = random.Random(seed)
    stalls = 0
    while live:
        g = rnd.choice(live)
        before = list(prog)
        try:
            next(gens[g])
        except StopIteration:
            live.remove(g)
        stalls = 0 if prog != before else stalls + 1
        assert stalls < 200000, "no block can make progress"
    return np.max(np.abs(x - ref))


@pytest.mark.parametrize("shape", [(5, 4, 6), (1, 7, 9), (8, 1, 5), (3, 2, 13), (6, 5, 1)])
@pytest.mark.parametrize("G", [1, 2, 3, 7])
@pytest.mark.parametrize("dirs", [(False,), (True,), (False, False, False), (False, True, False, True),
                                  (True, True, False)])
def test_gs27_plane_lagged_schedule_equals_sequential_sweeps(shape, G, dirs):
    assert _model_gs27p(shape, G, list(dirs), seed=hash((shape, G, dirs)) % 9973) < 1e-12


@pytest.mark.parametrize("PUB", [1, 2])
@pytest.mark.parametrize("lag", [4, 5])
def test_gs27_plane_lagged_kernel_parameters(PUB, lag):
    # the kernel publishes after every rem step and, loading each step's
    # operands a step ahead, waits for one rem more than the data needs
    for shape, G, dirs in (((7, 5, 11), 3, (False, False, True)), ((4, 9, 6), 2, (True, False, False))):
        assert _model_gs27p(shape, G, list(dirs), seed=17 * PUB + lag, PUB=PUB, lag=lag) < 1e-12


@pytest.mark.parametrize("kw", [dict(lag=3), dict(drop_old_side=True)])
def test_gs27p_model_detects_a_weakened_wait(kw):
    # one plane per block, so that no block's own earlier planes imply the
    # old-side wait
    errs = [_model_gs27p((6, 4, 9), 9, [False, False, True], seed=s, **kw) for s in range(6)]
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


# ---------------------------------------------------------------- 7-point pencils

def _model_gsp(shape, PY, PZ, W, dirs, seed, CH=3, PF=2, PFO=3, short_need=0, drop_old_side=False):
    """The pencil schedule of the 7-point Gauss-Seidel kernel (hs_gsp.cu,
    k_gsp).  A warp owns PY x PZ x-lines (lane = jl + PY kl) and sweeps them
    two nodes (a pair) per substep, lane (jl, kl) on sweep-frame pair u - D at
    substep u, D = jl + kl in the sweep's mirrored frame.  Neighbour lines of
    the pencil come from the lanes' registers as shuffles (new side: the
    neighbour's last computed pair; old side: the neighbour's next old pair);
    lines of other pencils from global memory, loaded PF substeps ahead, after
    waiting (per chunk of CH substeps) until the new-side pencils have
    published enough pairs of this sweep and the old-side pencils of the
    previous one.  Own-line old values are loaded PFO substeps ahead.  Stores
    become visible to other warps only at the chunk's publish; a load of
    another warp's line must see published data that nobody rewrites before
    the load is used.  Returns (model result, sequential result)."""
    nx, ny, nz = shape
    nJ, nK = -(-ny // PY), -(-nz // PZ)
    NP, NQ, Dmax = nJ * nK, -(-nx // 2), (PY - 1) + (PZ - 1)
    NU = NQ + Dmax
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(-1, 1, (nx, ny, nz))
    bD = rng.uniform(-1, 1, (nx, ny, nz))
    cxl, cxu, cyl, cyu, czl, czu = rng.uniform(0.02, 0.16, 6)

    def at(x, i, j, k):
        return x[i, j, k] if 0 <= i < nx and 0 <= j < ny and 0 <= k < nz else 0.0

    # sequential reference: the same two-part update, old side then new side
    ref = x0.copy()
    for bw in dirs:
        rng_k = range(nz - 1, -1, -1) if bw else range(nz)
        for k in rng_k:
            for j in (range(ny - 1, -1, -1) if bw else range(ny)):
                for i in (range(nx - 1, -1, -1) if bw else range(nx)):
                    s = 1 if bw else -1          # step towards the new side
                    ox, nxv = at(ref, i - s, j, k), at(ref, i + s, j, k)
                    oy, nyv = at(ref, i, j - s, k), at(ref, i, j + s, k)
                    oz, nzv = at(ref, i, j, k - s), at(ref, i, j, k + s)
                    co = (cxl, cyl, czl) if bw else (cxu, cyu, czu)
                    cn = (cxu, cyu, czu) if bw else (cxl, cyl, czl)
                    y = co[0] * ox + bD[i, j, k]
                    y = co[1] * oy + y
                    y = co[2] * oz + y
                    y = cn[0] * nxv + y
                    y = cn[1] * nyv + y
                    y = cn[2] * nzv + y
                    ref[i, j, k] = y

    X = x0.copy()                 # globally visible values
    owner = {}                    # address -> warp that last stored it
    pend = {}                     # warp -> {address: value} stored, not yet published
    stamp = {}                    # address -> count of stores issued
    prog = [0] * NP
    state = {"stores": 0}

    def store(w, addr, v):
        pend[w][addr] = v
        stamp[addr] = stamp.get(addr, 0) + 1
        owner[addr] = w

    def load(w, addr):
        # (value, address, stamp at issue): own pending stores are seen in
        # program order; another warp's unpublished store is a hazard
        if addr in pend[w]:
            return (pend[w][addr], addr, stamp.get(addr, 0))
        for w2, pe in pend.items():
            assert w2 == w or addr not in pe, "read of another warp's unpublished store at %s" % (addr,)
        return (X[addr], addr, stamp.get(addr, 0))

    def use(w, ld):
        v, addr, st0 = ld
        if addr is not None and owner.get(addr, w) != w:
            assert stamp.get(addr, 0) == st0, "value at %s rewritten while in flight" % (addr,)
        return v

    ZERO = (0.0, None, 0)

    def warp(w):
        pend[w] = {}
        per = -(-NP // W)                       # consecutive pencils per warp
        mine = list(range(w * per, min(NP, (w + 1) * per)))
        for t, bw in enumerate(dirs):
            for p in (reversed(mine) if bw else mine):
                J, K = p % nJ, p // nJ
                s = 1 if bw else -1                      # step towards the new side
                newn = [(J + s, K), (J, K + s)]
                oldn = [(J - s, K), (J, K - s)]
                newp = [q[0] + nJ * q[1] for q in newn if 0 <= q[0] < nJ and 0 <= q[1] < nK]
                oldp = [q[0] + nJ * q[1] for q in oldn if 0 <= q[0] < nJ and 0 <= q[1] < nK]
                same_dir = t > 0 and dirs[t - 1] == bw
                lanes = []
                for l in range(PY * PZ):
                    jl, kl = l % PY, l // PY
                    jm, km = (PY - 1 - jl, PZ - 1 - kl) if bw else (jl, kl)
                    j, k = J * PY + jl, K * PZ + kl
                    lanes.append(dict(jl=jl, kl=kl, jm=jm, km=km, D=jm + km, j=j, k=k,
                                      valid=j < ny and k < nz))

                def pos(qq):
                    # sweep-frame pair qq -> (first, second) x positions, None outside
                    if qq < 0 or qq >= NQ:
                        return (None, None)
                    q = NQ - 1 - qq if bw else qq
                    a, b = (2 * q + 1, 2 * q) if bw else (2 * q, 2 * q + 1)
                    return (a if a < nx else None, b if b < nx else None)

                def ld_pair(wq, qq, j, k):
                    if not (0 <= j < ny and 0 <= k < nz):
                        return (ZERO, ZERO)
                    a, b = pos(qq)
                    return tuple(load(wq, (i, j, k)) if i is not None else ZERO for i in (a, b))

                # registers: per lane dicts keyed by sweep-frame pair
                for L in lanes:
                    L["O"], L["B"], L["NY"], L["NZ"], L["OY"], L["OZ"] = {}, {}, {}, {}, {}, {}
                    L["last"] = (0.0, 0.0)

                def issue(L, u):
                    # loads issued at substep u (prologue: u < 0 covers the window)
                    if not L["valid"]:
                        return
                    j, k, D = L["j"], L["k"], L["D"]
                    qo = u - D + PFO                     # own old pair
                    if 0 <= qo < NQ:
                        L["O"][qo] = ld_pair(w, qo, j, k)
                        a, b = pos(qo)
                        L["B"][qo] = tuple((bD[i, j, k], None, 0) if i is not None else ZERO for i in (a, b))
                    qb = u - D + PF                      # pencil-boundary pairs
                    if 0 <= qb < NQ:
                        if L["jm"] == 0:
                            L["NY"][qb] = ld_pair(w, qb, j + s, k)
                        if L["km"] == 0:
                            L["NZ"][qb] = ld_pair(w, qb, j, k + s)
                        if L["jm"] == PY - 1:
                            L["OY"][qb] = ld_pair(w, qb, j - s, k)
                        if L["km"] == PZ - 1:
                            L["OZ"][qb] = ld_pair(w, qb, j, k - s)

                def ready(c):
                    need = min(NQ, (c + 1) * CH + PF - short_need)
                    if any(prog[q] < t * NQ + need for q in newp):
                        return False
                    if t > 0 and not drop_old_side:
                        tgt = (t - 1) * NQ + need if same_dir else t * NQ
                        if any(prog[q] < tgt for q in oldp):
                            return False
                    return prog[p] >= t * NQ                 # the pencil's previous sweep

                nchunks = -(-NU // CH)
                for c in range(nchunks):
                    while not ready(c):
                        yield False
                    if c == 0:
                        for L in lanes:
                            for u in range(-max(PF, PFO), 0):
                                issue(L, u)
                    for u in range(c * CH, min((c + 1) * CH, NU)):
                        snap = [dict(last=L["last"]) for L in lanes]
                        for L in lanes:
                            # the old pair a lane processes next: its new-side
                            # neighbour line processes that pair now
                            qn = u - L["D"] + 1
                            L["onx_shared"] = L["O"].get(qn, (ZERO, ZERO)) if L["valid"] else (ZERO, ZERO)
                        for idx, L in enumerate(lanes):
                            qq = u - L["D"]
                            if not (L["valid"] and 0 <= qq < NQ):
                                continue
                            jl, kl = L["jl"], L["kl"]
                            # lane offsets of the new-side / old-side neighbour lines
                            dyn = 1 if bw else -1
                            if L["jm"] == 0:
                                ny_ = tuple(use(w, v) for v in L["NY"].pop(qq))
                            else:
                                ny_ = snap[idx + dyn]["last"]
                            if L["km"] == 0:
                                nz_ = tuple(use(w, v) for v in L["NZ"].pop(qq))
                            else:
                                nz_ = snap[idx + dyn * PY]["last"]
                            if L["jm"] == PY - 1:
                                oy = tuple(use(w, v) for v in L["OY"].pop(qq))
                            else:
                                oy = tuple(use(w, v) for v in lanes[idx - dyn]["onx_shared"])
                            if L["km"] == PZ - 1:
                                oz = tuple(use(w, v) for v in L["OZ"].pop(qq))
                            else:
                                oz = tuple(use(w, v) for v in lanes[idx - dyn * PY]["onx_shared"])
                            ocur = tuple(use(w, v) for v in L["O"].pop(qq))
                            onx = tuple(use(w, v) for v in L["O"].get(qq + 1, (ZERO, ZERO)))
                            bq = tuple(v[0] for v in L["B"].pop(qq))
                            co = (cxl, cyl, czl) if bw else (cxu, cyu, czu)
                            cn = (cxu, cyu, czu) if bw else (cxl, cyl, czl)
                            a, b = pos(qq)
                            # first node: x old = this pair's second, x new = previous pair's second
                            y = co[0] * ocur[1] + bq[0]
                            y = co[1] * oy[0] + y
                            y = co[2] * oz[0] + y
                            y = cn[0] * L["last"][1] + y
                            y = cn[1] * ny_[0] + y
                            na = cn[2] * nz_[0] + y if a is not None else 0.0
                            y = co[0] * onx[0] + bq[1]
                            y = co[1] * oy[1] + y
                            y = co[2] * oz[1] + y
                            y = cn[0] * na + y
                            y = cn[1] * ny_[1] + y
                            nb = cn[2] * nz_[1] + y if b is not None else 0.0
                            L["newlast"] = (na, nb)
                            j, k = L["j"], L["k"]
                            if a is not None:
                                store(w, (a, j, k), na)
                            if b is not None:
                                store(w, (b, j, k), nb)
                        for L in lanes:
                            if "newlast" in L:
                                L["last"] = L.pop("newlast")
                            issue(L, u)
                        yield True
                    # publish: stores become visible, then the progress count
                    for addr, v in pend[w].items():
                        X[addr] = v
                    pend[w].clear()
                    u_end = min((c + 1) * CH, NU)
                    prog[p] = t * NQ + max(0, min(NQ, u_end - Dmax))
                    yield True

    gens = {w: warp(w) for w in range(W)}
    rr = random.Random(seed)
    live = set(gens)
    stall = 0
    while live:
        w = rr.choice(sorted(live))
        try:
            moved = next(gens[w])
        except StopIteration:
            live.discard(w)
            stall = 0
            continue
        stall = 0 if moved else stall + 1
        assert stall < 200 * len(live) + 1000, "no warp can proceed (deadlock)"
    return X, ref


@pytest.mark.parametrize("shape,PY,PZ,W,dirs", [
    ((9, 7, 5), 4, 2, 3, [0, 0, 0]),
    ((8, 9, 6), 4, 2, 100, [0, 0]),
    ((11, 6, 7), 2, 2, 4, [1, 1]),
    ((7, 5, 9), 4, 2, 2, [0, 1, 0, 1]),
    ((10, 8, 4), 4, 4, 1, [0, 0, 1]),
    ((5, 3, 3), 8, 4, 5, [0, 1]),
])
def test_gsp_pencil_schedule_equals_sequential_sweeps(shape, PY, PZ, W, dirs):
    for seed in range(3):
        X, ref = _model_gsp(shape, PY, PZ, W, dirs, seed)
        assert np.array_equal(X, ref), (shape, PY, PZ, W, dirs, seed, np.max(np.abs(X - ref)))


@pytest.mark.parametrize("kw", [dict(short_need=2, CH=1), dict(drop_old_side=True)])
def test_gsp_model_detects_a_weakened_wait(kw):
    # waiting for two pairs too few (with one substep per chunk, so that the
    # producers publish every pair; a published count is that of the pencil's
    # last line, PZ - 1 = 1 pair behind the line a y-boundary lane reads, so
    # one pair less is still safe), or not at all on the old side, must show
    # up as a wrong value or a hazard in some interleaving
    caught = 0
    for seed in range(12):
        try:
            X, ref = _model_gsp((9, 8, 6), 4, 2, 6, [0, 0, 0], seed, **kw)
            caught += int(not np.array_equal(X, ref))
        except AssertionError:
            caught += 1
    assert caught > 0


# ---------------------------------------------------------------- tile-plane tables

def _gs_tables_closed_form(a, b, c):
    """The device's tile-plane tables (hs_gs.cu, k_gs_plane_off and
    k_gs_plane_tiles) transcribed: offsets from the count of tiles (I, J) of one
    layer on plane u, and each tile's rank inside its plane."""
    def n2(u):
        if u < 0:
            return 0
        lo, hi = max(0, u - b + 1), min(u, a - 1)
        return hi - lo + 1 if hi >= lo else 0
    P = a + b + c - 2
    off = [sum(n2(sp - k) for sp in range(q) for k in range(c)) for q in range(P + 1)]
    tiles = [None] * (a * b * c)
    for t in range(a * b * c):
        I, J, K = t % a, (t // a) % b, t // (a * b)
        S = I + J + K
        rank = sum(n2(S - k) for k in range(K)) + sum(1 for j in range(J) if 0 <= S - K - j < a)
        tiles[off[S] + rank] = t
    return off, tiles


def _gs_tables_counting_sort(a, b, c):
    P = a + b + c - 2
    # plain counting sort by plane, ids increasing within a plane
    planes = {}
    for t in range(a * b * c):
        I, J, K = t % a, (t // a) % b, t // (a * b)
        planes.setdefault(I + J + K, []).append(t)
    off, tiles, acc = [], [], 0
    for s in range(P + 1):
        off.append(acc)
        acc += len(planes.get(s, []))
        tiles += planes.get(s, [])
    return off, tiles


@pytest.mark.parametrize("shape", [(1, 1, 1), (8, 32, 32), (3, 5, 2), (1, 7, 4), (6, 1, 9), (4, 4, 4), (2, 16, 1)])
def test_gs_tile_tables_closed_form_equals_counting_sort(shape):
    off, tiles = _gs_tables_closed_form(*shape)
    off2, tiles2 = _gs_tables_counting_sort(*shape)
    assert off == off2 and tiles == tiles2


# ---------------------------------------------------------------- 2-D GS on a cluster

def _gs2dc_work(nx, ny, C, nsw, bw, s, i):
    """(sweep, row) pairs CTA by CTA for column i at step s, with the index
    arithmetic of k_gs2dc (rows split over C CTAs, the t range of each CTA's
    rows in the sweep's frame)."""
    R = -(-ny // C)
    out = []
    for rank in range(C):
        r0, r1 = min(ny, rank * R), min(ny, rank * R + R)
        f0, f1 = (ny - r1, ny - r0) if bw else (r0, r1)
        if f1 <= f0:
            continue
        t_lo = max(0, (s - i - f1 + 2) >> 1)
        t_hi = min(nsw - 1, (s - i - f0) >> 1)
        for t in range(t_lo, t_hi + 1):
            r = s - 2 * t - i
            if f0 <= r < f1:
                jj = ny - 1 - r if bw else r
                assert r0 <= jj < r1
                out.append((t, r))
    return out


@pytest.mark.parametrize("nx,ny,C,nsw", [(8, 16, 8, 3), (5, 17, 8, 4), (12, 40, 8, 1), (3, 23, 4, 6), (128, 128, 8, 5)])
@pytest.mark.parametrize("bw", [False, True])
def test_gs2d_cluster_rows_cover_every_sweep_row_once(nx, ny, C, nsw, bw):
    # at every step, the CTAs together handle exactly the (sweep, row) pairs
    # of the one-block wavefront: row s - 2t - i of sweep t, for every sweep
    # whose diagonal crosses column i
    nsteps = (nx + ny - 2) + 1 + 2 * (nsw - 1)
    seen = set()
    for s in range(nsteps):
        for i in range(nx):
            got = _gs2dc_work(nx, ny, C, nsw, bw, s, i)
            want = [(t, s - 2 * t - i) for t in range(nsw) if 0 <= s - 2 * t - i < ny]
            assert sorted(got) == sorted(want), (s, i, got, want)
            for t, r in got:
                assert (t, r, i) not in seen
                seen.add((t, r, i))
    assert len(seen) == nsw * nx * ny
