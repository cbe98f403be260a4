"""CPU models of the streamed single-right-hand-side kernels (csrc/stream.cu).

1. Addressing: the kernels' index arithmetic, restated here, replayed for
   every tile of whole grids -- every tensor-map box must lie inside its
   map with its x coordinate on 16 bytes, every partial-sum index inside
   the buffer, every Step-2 read inside its node's partials and on a slot
   that the CTA owning it wrote, every node's arrivals adding up to its
   tile count -- over the geometry the library reports for the handle
   (hmat_info of a host-only build).
2. Barrier protocol: the producer / consumer / weights-warp protocol of the
   two kernels over mbarriers with the hardware's parity rule (a wait on
   parity P passes while the barrier's current phase parity differs from
   P), run under random schedules: it must never deadlock, and no wait may
   pass on a phase other than the one it means (phase aliasing).

Sizes are those of the tests and workloads (the kernels' parameters follow
from the geometry as the launch code computes them)."""
import random

import pytest

import workloads as w

KB = 1024
TILE_E = 256                     # expand tile (kExpandStreamTile)


@pytest.fixture(scope="module")
def hm():
    from paper_2008_12441_gb300 import _build
    _build.build()
    from paper_2008_12441_gb300 import hmat
    return hmat


# ------------------------------------------------------------------ geometry
def geometry(info, tile_cap=256):
    """Level layout as the builder lays it out (node sums, then per-tile
    partials of the levels whose nodes span several project tiles)."""
    d, L, Np = info.d, info.depth, info.padded_N
    s = (1 << d) - 1
    nf = info.lowrank_levels
    tile = info.leaf_slots
    while tile * 2 <= tile_cap and tile * 2 <= Np:
        tile *= 2
    lv, t_off = {}, 0
    for l in range(1, nf + 1):
        n = Np >> (d * l)
        r = info.rank_per_level[l]
        lv[l] = dict(n=n, nodes=1 << (d * l), r=r, sr=s * r,
                     nsub=n // tile if n > tile else 1)
    for l in range(1, nf + 1):
        g = lv[l]
        g["fin"] = t_off
        t_off += g["nodes"] * g["sr"]
        if g["nsub"] > 1:
            g["part"] = t_off
            t_off += (Np // tile) * g["sr"]
    G = (1 << d) * info.leaf_slots
    return dict(d=d, s=s, nf=nf, Np=Np, tile=tile, lv=lv, T=t_off, G=G)


def largest_divisor_at_most(v, cap):
    for b in range(min(v, cap), 1, -1):
        if v % b == 0:
            return b
    return 1


def replay(g, es, sms=152):
    """Every address the two kernels form, checked; returns the faults."""
    bad = []
    tile, Np, s = g["tile"], g["Np"], g["s"]
    RB = max(1, min(32, 24 * KB // (tile * es)))
    stages = []
    for l, L in g["lv"].items():
        if L["r"] == 0:
            continue
        L["rb"] = largest_divisor_at_most(L["sr"], RB)
        L["rbu"] = largest_divisor_at_most(L["sr"], max(1, min(64, 16 * KB // (TILE_E * es))))
        stages += [(l, c, L["rb"]) for c in range(0, L["sr"], L["rb"])]
    # project: tiles of CTA c are [c R, c R + R)
    ntile = Np // tile
    R = -(-ntile // sms)
    for t in range(ntile):
        p0 = t * tile
        if p0 + tile > Np:
            bad.append(("x copy", t))
        for l, c0, rows in stages:
            L = g["lv"][l]
            node = p0 // L["n"]
            inoff = p0 - node * L["n"]
            if not (0 <= inoff and inoff + tile <= L["n"] and (inoff * es) % 16 == 0):
                bad.append(("V box x", l, t))
            if node * L["sr"] + c0 + rows > L["nodes"] * L["sr"] or rows > RB:
                bad.append(("V box y", l, t))
            base = L["part"] + t * L["sr"] if L["nsub"] > 1 else L["fin"] + node * L["sr"]
            if not (0 <= base + c0 and base + c0 + rows <= g["T"]):
                bad.append(("T store", l, t))
    grid = -(-ntile // R)
    assert grid <= sms
    # Step 2 at the end of the project kernel.  CTA c: for each node j it
    # touches, the sum of its tiles [ta, tb) goes to the slot of tile ta and
    # it adds tb - ta to the node's counter; the completing CTA reads the
    # slot max(c R, j nsub) of every CTA c in [j nsub / R, ((j+1) nsub - 1) / R].
    for l, L in g["lv"].items():
        if L["nsub"] <= 1 or L["r"] == 0:
            continue
        nsub, sr = L["nsub"], L["sr"]
        written = {}                 # node -> {slot tile: CTA}
        arrivals = [0] * L["nodes"]
        for c in range(grid):
            tb_, te_ = c * R, min(c * R + R, ntile)
            for j in range(tb_ // nsub, (te_ - 1) // nsub + 1):
                ta, tb = max(tb_, j * nsub), min(te_, (j + 1) * nsub)
                if not (ta < tb and j < L["nodes"]):
                    bad.append(("step-2 node range", l, c, j))
                    continue
                for t in range(ta, tb):
                    if not (0 <= L["part"] + t * sr and L["part"] + t * sr + sr <= g["T"]):
                        bad.append(("step-2 partial read", l, t))
                written.setdefault(j, {})[ta] = c
                arrivals[j] += tb - ta
        for j in range(L["nodes"]):
            if arrivals[j] != nsub:
                bad.append(("step-2 arrivals", l, j, arrivals[j]))
            c0, c1 = j * nsub // R, ((j + 1) * nsub - 1) // R
            reads = {max(c * R, j * nsub): c for c in range(c0, c1 + 1)}
            if reads != written.get(j):
                bad.append(("step-2 node read", l, j))
    # expand: D boxes, U boxes, node-sum reads of the target's siblings
    G, nc = g["G"], s + 1
    rbd = largest_divisor_at_most(G, max(1, min(64, 16 * KB // (TILE_E * es))))
    for t in range(Np // TILE_E):
        e0 = t * TILE_E
        g0 = e0 // G
        for c0 in range(0, G, rbd):
            if e0 - g0 * G + TILE_E > G or g0 * G + c0 + rbd > (Np // G) * G:
                bad.append(("D box", t))
        for l, L in g["lv"].items():
            if L["r"] == 0:
                continue
            i = e0 // L["n"]
            x = e0 - i * L["n"]
            if x + TILE_E > L["n"] or (x * es) % 16:
                bad.append(("U box x", l, t))
            if i * L["sr"] + L["sr"] > L["nodes"] * L["sr"]:
                bad.append(("U box y", l, t))
            ci = i % nc
            for col in range(L["sr"]):
                q, cr = divmod(col, L["r"])
                cj = q if q < ci else q + 1
                j = i - ci + cj
                qv = ci if ci < cj else ci - 1
                idx = L["fin"] + j * L["sr"] + qv * L["r"] + cr
                if not (L["fin"] <= idx < L["fin"] + L["nodes"] * L["sr"]) or j // nc != i // nc:
                    bad.append(("T read", l, t, col))
    return bad


@pytest.mark.parametrize("d,n,r,es", [(2, 64, 4, 4), (2, 128, 16, 4), (2, 256, 4, 4), (2, 256, 16, 2),
                                      (2, 128, 8, 8), (3, 16, 32, 4), (3, 32, 4, 4), (3, 32, 8, 1)])
def test_streamed_addressing_in_bounds(hm, d, n, r, es):
    opts = hm.hmat_default_opts(device=-1, method=2, seed=5, prec=1)
    h = hm.hmat_build(w.grid_points(n, d), 2, 64, r, 0.0, opts)
    try:
        g = geometry(hm.hmat_info(h))
    finally:
        hm.hmat_destroy(h)
    assert all(L["n"] >= g["tile"] for L in g["lv"].values())
    assert replay(g, es) == []


# ------------------------------------------------------------ barrier model
class Bar:
    """mbarrier: `count` arrivals complete a phase; waits use the parity rule."""

    def __init__(self, count):
        self.count, self.pending, self.phase = count, count, 0

    def arrive(self):
        self.pending -= 1
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count


def wait(bar, parity, meant):
    """A wait on `parity` that means completion number `meant` (0-based)."""
    return ("wait", bar, parity, meant)


def landing(bar):
    """An asynchronous copy in flight: it arrives on `bar` whenever the
    scheduler picks it, in any order relative to other copies and waits."""
    bar.arrive()
    return
    yield


def run(actors, rng):
    """Random schedule of the actors; an actor may yield ("spawn", gen) to
    start an asynchronous copy (a new actor that is always ready)."""
    actors = dict(actors)
    cur = {}
    spawned = [0]

    def advance(k):
        while True:
            v = next(actors[k], None)
            if v is not None and v[0] == "spawn":
                spawned[0] += 1
                name = f"copy{spawned[0]}"
                actors[name] = v[1]
                cur[name] = ("ready",)
                continue
            cur[k] = v
            return

    for k in list(actors):
        advance(k)
    while True:
        live = [k for k, v in cur.items() if v is not None]
        if not live:
            return "ok"
        ready = []
        for k in live:
            if cur[k][0] == "ready":
                ready.append(k)
                continue
            _, bar, parity, meant = cur[k]
            if (bar.phase & 1) != parity:
                # passes: it must be the phase it means (no aliasing)
                if bar.phase != meant + 1:
                    return f"aliased wait of {k}: phase {bar.phase}, meant {meant}"
                ready.append(k)
        if not ready:
            return "deadlock"
        advance(rng.choice(ready))


def project_model(ntl, Q, S=8, XB=8, ahead=6, skip_xempty=False):
    """project_stream_kernel: one producer; consumer warp w owns ring slot w
    (S slots, S warps) and takes stages w, w + S, ...; x of tile u goes to
    buffer u % XB `ahead` tiles early, once the tile that used the buffer
    has been consumed (one arrival per stage), and a tile's stages are
    issued after its x has landed.  Consumers never wait on the x barriers:
    a stage they read must find its tile's x in the buffer (checked)."""
    full = [Bar(1) for _ in range(S)]
    empty = [Bar(1) for _ in range(S)]
    xfull = [Bar(32) for _ in range(XB)]
    xempty = [Bar(Q) for _ in range(XB)]
    xtile = [None] * XB              # tile whose x the buffer holds

    def producer():
        def load_x(u):
            b = u % XB
            if u >= XB and not skip_xempty:
                yield wait(xempty[b], ((u // XB) - 1) & 1, u // XB - 1)
            xtile[b] = u
            yield ("spawn", landing(xfull[b]))        # the bulk copy
            for _ in range(31):
                xfull[b].arrive()
        for u in range(min(ahead, ntl)):
            yield from load_x(u)
        for u in range(ntl):
            if u + ahead < ntl:
                yield from load_x(u + ahead)
            yield wait(xfull[u % XB], (u // XB) & 1, u // XB)
            for q in range(Q):
                g = u * Q + q
                if g >= S:
                    yield wait(empty[g % S], (g // S - 1) & 1, g // S - 1)
                yield ("spawn", landing(full[g % S]))
        total = ntl * Q
        for g in range(max(total - S, 0), total):
            yield wait(full[g % S], (g // S) & 1, g // S)
        for u in range(max(ntl - XB, 0), ntl):
            yield wait(xfull[u % XB], (u // XB) & 1, u // XB)

    def consumer(w):
        for g in range(w, ntl * Q, S):
            yield wait(full[w], (g // S) & 1, g // S)
            if xtile[(g // Q) % XB] != g // Q:
                raise AssertionError(f"stage {g} read x of tile {xtile[(g // Q) % XB]}")
            empty[w].arrive()
            xempty[(g // Q) % XB].arrive()

    actors = {"producer": producer()}
    actors.update({f"consumer{i}": consumer(i) for i in range(S)})
    return actors


def expand_model(ntl, Q, S, groups=4, by_tile=False):
    """expand_stream_kernel: stage g (tile g // Q, stage g % Q) goes to group
    g mod 4 (by_tile: the planted mistake of an earlier version, stage q of
    every tile to group q mod 4, so that a ring slot's uses change groups
    from tile to tile); the boxes land asynchronously, in any order."""
    full = [Bar(1) for _ in range(S)]
    empty = [Bar(2) for _ in range(S)]
    wfull = [Bar(32) for _ in range(2)]
    wempty = [Bar(2 * groups) for _ in range(2)]
    rfull = [Bar(2 * groups) for _ in range(2)]
    rempty = [Bar(1) for _ in range(2)]

    def producer():
        for u in range(ntl):
            for q in range(Q):
                g = u * Q + q
                if g >= S:
                    yield wait(empty[g % S], (g // S - 1) & 1, g // S - 1)
                yield ("spawn", landing(full[g % S]))
        total = ntl * Q
        for g in range(max(total - S, 0), total):
            yield wait(full[g % S], (g // S) & 1, g // S)

    def weights():
        def combine(u):
            yield wait(rfull[u & 1], (u >> 1) & 1, u >> 1)
            rempty[u & 1].arrive()
        for u in range(ntl):
            xb = u & 1
            if u >= 2:
                yield wait(wempty[xb], ((u >> 1) - 1) & 1, (u >> 1) - 1)
            for _ in range(32):
                wfull[xb].arrive()
            if u >= 1:
                yield from combine(u - 1)
        if ntl >= 1:
            yield from combine(ntl - 1)

    def consumer(warp):
        grp = warp >> 1
        for u in range(ntl):
            xb = u & 1
            yield wait(wfull[xb], (u >> 1) & 1, u >> 1)
            q0 = grp if by_tile else (grp - u * Q) % groups
            for q in range(q0, Q, groups):
                g = u * Q + q
                yield wait(full[g % S], (g // S) & 1, g // S)
                empty[g % S].arrive()
            if u >= 2:
                yield wait(rempty[xb], ((u >> 1) - 1) & 1, (u >> 1) - 1)
            rfull[xb].arrive()
            wempty[xb].arrive()

    actors = {"producer": producer(), "weights": weights()}
    actors.update({f"consumer{i}": consumer(i) for i in range(2 * groups)})
    return actors


@pytest.mark.parametrize("ntl", [1, 2, 3, 7, 28])
@pytest.mark.parametrize("Q", [1, 2, 3, 5, 7, 8, 10, 12, 14, 15])
def test_project_protocol_no_deadlock_no_aliasing(ntl, Q):
    for seed in range(4):
        assert run(project_model(ntl, Q), random.Random(seed)) == "ok"


@pytest.mark.parametrize("ntl", [1, 2, 3, 7])
@pytest.mark.parametrize("Q,S", [(3, 4), (20, 12), (21, 12), (31, 12), (34, 12), (38, 12), (40, 12),
                                 (918, 4), (54, 8), (13, 8)])
def test_expand_protocol_no_deadlock_no_aliasing(ntl, Q, S):
    # the ring depth is a multiple of the four groups: each slot's uses all
    # belong to one group, which waits for them in order
    for seed in range(4):
        assert run(expand_model(ntl, Q, S), random.Random(seed)) == "ok"


def test_expand_model_catches_slots_changing_groups():
    """The assignment an earlier version used (stage q of each tile to group
    q mod 4) lets a slot's consecutive uses belong to different groups when
    the stage count is not a multiple of four; with asynchronous landings a
    group's wait can then pass on the slot's previous phase.  The model finds
    it (this is the mechanism of the two-second stage waits that were once
    seen, status 0x206)."""
    outs = [run(expand_model(ntl, Q, S, by_tile=True), random.Random(seed))
            for ntl, Q, S in [(3, 31, 12), (3, 34, 12), (2, 54, 5), (2, 5, 4)] for seed in range(12)]
    assert any(o.startswith("aliased") for o in outs)


def test_project_model_catches_an_early_x_overwrite():
    """Planted mistake: a producer that reloads an x buffer without waiting
    for the tile that used it to be consumed is caught by the model."""
    caught = 0
    for seed in range(8):
        try:
            run(project_model(28, 1, skip_xempty=True), random.Random(seed))
        except AssertionError:
            caught += 1
    assert caught > 0


def test_model_catches_a_planted_protocol_mistake():
    """The model is not vacuous: a producer that reuses a stage without
    waiting for it to be consumed lets a consumer's wait pass on the wrong
    phase."""
    def broken(ntl, Q, S):
        full = [Bar(1) for _ in range(S)]

        def producer():
            for g in range(ntl * Q):
                full[g % S].arrive()        # no wait on the stage's empty barrier
            yield wait(full[0], 0, 0)

        def consumer():
            for g in range(ntl * Q):
                yield wait(full[g % S], (g // S) & 1, g // S)

        return {"producer": producer(), "c0": consumer(), "c1": consumer()}
    outcomes = {run(broken(3, 5, 2), random.Random(s)) for s in range(4)}
    assert any(o != "ok" for o in outcomes)


# ------------------------------------------- tensor-core kernels (tc_matvec.cu)
def tc_project_model(tiles_per_node, nacc_l, t_begin, ntl, nchunk, cps, S, f8, kx=3, sr_ring=4,
                     seg=None):
    """tc_project_tma: producer (x chunks, V boxes; e4m3: raw boxes), MMA
    issuer (per-accumulator fresh / used / parity state), e4m3 converter
    warps, four epilogue warps (stand-ins for 128 arriving threads)."""
    nacc = sum(nacc_l)
    first = [sum(nacc_l[:i]) for i in range(len(nacc_l))]
    t_end = t_begin + ntl
    full = [Bar(4 if f8 else 1) for _ in range(S)]
    empty = [Bar(1) for _ in range(S)]
    xfull = [Bar(1) for _ in range(kx)]
    xempty = [Bar(1) for _ in range(kx)]
    afull = [Bar(1) for _ in range(nacc)]
    aempty = [Bar(4) for _ in range(nacc)]
    rfull = [Bar(1) for _ in range(sr_ring)]
    rempty = [Bar(4) for _ in range(sr_ring)]

    def flushes(li, t):
        # node end, range end, or (split storage) accumulation-segment end
        return (t == t_end - 1 or (t + 1) % tiles_per_node[li] == 0 or
                (seg is not None and (t + 1 - t_begin) % seg == 0))

    def producer():
        g = xc = 0
        for t in range(t_begin, t_end):
            for kc in range(0, nchunk, cps):
                xi = xc % kx
                if xc >= kx:
                    yield wait(xempty[xi], ((xc // kx) - 1) & 1, xc // kx - 1)
                xfull[xi].arrive()
                for li in range(len(nacc_l)):
                    for cb in range(nacc_l[li]):
                        if f8:
                            rs = g % sr_ring
                            if g >= sr_ring:
                                yield wait(rempty[rs], ((g // sr_ring) - 1) & 1, g // sr_ring - 1)
                            rfull[rs].arrive()
                        else:
                            s = g % S
                            if g >= S:
                                yield wait(empty[s], ((g // S) - 1) & 1, g // S - 1)
                            full[s].arrive()
                        g += 1
                xc += 1
        if f8:
            for q in range(max(g - sr_ring, 0), g):
                yield wait(rfull[q % sr_ring], (q // sr_ring) & 1, q // sr_ring)
        else:
            for q in range(max(g - S, 0), g):
                yield wait(full[q % S], (q // S) & 1, q // S)
        for q in range(max(xc - kx, 0), xc):
            yield wait(xfull[q % kx], (q // kx) & 1, q // kx)

    def mma():
        fresh, used, par = (1 << nacc) - 1, 0, 0
        nflush = [0] * nacc
        g = xc = 0
        for t in range(t_begin, t_end):
            for kc in range(0, nchunk, cps):
                xi = xc % kx
                yield wait(xfull[xi], (xc // kx) & 1, xc // kx)
                for ai in range(nacc):
                    s, bit = g % S, 1 << ai
                    if kc == 0 and (fresh & used & bit):
                        yield wait(aempty[ai], ((par >> ai) & 1) ^ 1, nflush[ai] - 1)
                    yield wait(full[s], (g // S) & 1, g // S)
                    if kc == 0:
                        fresh &= ~bit
                    empty[s].arrive()
                    g += 1
                xempty[xi].arrive()
                xc += 1
            for li in range(len(nacc_l)):
                if flushes(li, t):
                    for ai in range(first[li], first[li] + nacc_l[li]):
                        afull[ai].arrive()
                        fresh |= 1 << ai
                        used |= 1 << ai
                        par ^= 1 << ai
                        nflush[ai] += 1

    def converter():
        g = 0
        for t in range(t_begin, t_end):
            for kc in range(0, nchunk, cps):
                for ai in range(nacc):
                    rs, s = g % sr_ring, g % S
                    yield wait(rfull[rs], (g // sr_ring) & 1, g // sr_ring)
                    if g >= S:
                        yield wait(empty[s], ((g // S) - 1) & 1, g // S - 1)
                    rempty[rs].arrive()
                    full[s].arrive()
                    g += 1

    def epilogue():
        n = [0] * nacc
        for t in range(t_begin, t_end):
            for li in range(len(nacc_l)):
                if flushes(li, t):
                    for ai in range(first[li], first[li] + nacc_l[li]):
                        yield wait(afull[ai], n[ai] & 1, n[ai])
                        aempty[ai].arrive()
                        n[ai] += 1

    actors = {"producer": producer(), "mma": mma()}
    actors.update({f"epilogue{i}": epilogue() for i in range(4)})
    if f8:
        actors.update({f"converter{i}": converter() for i in range(4)})
    return actors


def tc_expand_model(chunks, has_rank, t_begin, ntl, S, f8, sr_ring=4):
    """tc_expand_tma: chunks[0] near-field stages, chunks[l] stages of level
    l per tile; double-buffered accumulators; e4m3: raw U boxes converted
    by four warps that also release every stage."""
    full = [Bar(5 if f8 else 1) for _ in range(S)]
    empty = [Bar(1) for _ in range(S)]
    afull = [Bar(1) for _ in range(2)]
    aempty = [Bar(4) for _ in range(2)]
    rfull = [Bar(1) for _ in range(sr_ring)]
    rempty = [Bar(4) for _ in range(sr_ring)]
    segs = [(0, chunks[0])] + [(l, chunks[l]) for l in range(len(chunks) - 1, 0, -1) if has_rank[l]]

    def producer():
        g = gr = 0
        for t in range(ntl):
            for l, nch in segs:
                for _ in range(nch):
                    s = g % S
                    if g >= S:
                        yield wait(empty[s], ((g // S) - 1) & 1, g // S - 1)
                    if f8 and l > 0:
                        rs = gr % sr_ring
                        if gr >= sr_ring:
                            yield wait(rempty[rs], ((gr // sr_ring) - 1) & 1, gr // sr_ring - 1)
                        rfull[rs].arrive()
                        gr += 1
                    full[s].arrive()
                    g += 1
        if f8:
            for q in range(max(gr - sr_ring, 0), gr):
                yield wait(rfull[q % sr_ring], (q // sr_ring) & 1, q // sr_ring)
        for q in range(max(g - S, 0), g):
            yield wait(full[q % S], (q // S) & 1, q // S)

    def mma():
        g = 0
        for u in range(ntl):
            ab = u & 1
            if u >= 2:
                yield wait(aempty[ab], ((u >> 1) - 1) & 1, (u >> 1) - 1)
            for l, nch in segs:
                for _ in range(nch):
                    yield wait(full[g % S], (g // S) & 1, g // S)
                    empty[g % S].arrive()
                    g += 1
            afull[ab].arrive()

    def converter():
        g = gr = 0
        for t in range(ntl):
            for l, nch in segs:
                for _ in range(nch):
                    s = g % S
                    if g >= S:
                        yield wait(empty[s], ((g // S) - 1) & 1, g // S - 1)
                    if l > 0:
                        yield wait(rfull[gr % sr_ring], (gr // sr_ring) & 1, gr // sr_ring)
                        rempty[gr % sr_ring].arrive()
                        gr += 1
                    full[s].arrive()
                    g += 1

    def epilogue():
        for u in range(ntl):
            yield wait(afull[u & 1], (u >> 1) & 1, u >> 1)
            aempty[u & 1].arrive()

    actors = {"producer": producer(), "mma": mma()}
    actors.update({f"epilogue{i}": epilogue() for i in range(4)})
    if f8:
        actors.update({f"converter{i}": converter() for i in range(4)})
    return actors


# geometries of the bench's multi-RHS workloads and of the 2D default:
# (tiles of 256 slots per node per level, accumulator blocks per level)
TC_PROJECT_GEOMETRIES = {
    "3d-64^3-r32": ([128, 16, 2], [2, 2, 2]),
    "2d-512^2-r16": ([256, 64, 16, 4, 1], [1] * 5),
    "2d-1024^2-r16": ([1024, 256, 64, 16, 4, 1], [1] * 6),
}


@pytest.mark.parametrize("geo", sorted(TC_PROJECT_GEOMETRIES))
@pytest.mark.parametrize("cps,S", [(1, 4), (2, 4), (2, 13), (1, 32), (4, 4), (4, 6)])
@pytest.mark.parametrize("f8", [False, True])
@pytest.mark.parametrize("seg", [None, 4])
def test_tc_project_protocol(geo, cps, S, f8, seg):
    tpn, nacc_l = TC_PROJECT_GEOMETRIES[geo]
    # ranges of seven tiles starting anywhere, and short last ranges; e4m3
    # raw rings of 4 and of 12 slots
    for t_begin, ntl in [(0, 7), (7, 7), (126, 7), (1015, 7), (0, 1), (5, 2), (27, 27)]:
        for seed in range(2):
            for sr in ((4, 12) if f8 else (4,)):
                out = run(tc_project_model(tpn, nacc_l, t_begin, ntl, 4, cps, S, f8, seg=seg, sr_ring=sr,
                                           kx=2 if cps == 4 else 3),
                          random.Random(seed))
                assert out == "ok", (geo, cps, S, f8, t_begin, ntl, sr, out)


@pytest.mark.parametrize("chunks", [[8, 4, 4, 4], [4, 1, 1, 1, 1, 1], [2, 1]])
@pytest.mark.parametrize("S", [3, 6, 10])
@pytest.mark.parametrize("f8", [False, True])
def test_tc_expand_protocol(chunks, S, f8):
    has_rank = [True] * len(chunks)
    for ntl in (1, 2, 3, 14):
        for seed in range(2):
            for sr in ((4, 8) if f8 else (4,)):
                out = run(tc_expand_model(chunks, has_rank, 0, ntl, S, f8, sr_ring=sr), random.Random(seed))
                assert out == "ok", (chunks, S, f8, ntl, sr, out)


def prep_elem(n, k):
    """Element of (row n, column k) in a prepared B operand region: 64 x 64
    chunks, 8 x 8 cores (the layout tc_xprep_kernel and tt_store write)."""
    return (k >> 6) * 4096 + (n >> 3) * 512 + ((k & 63) >> 3) * 64 + (n & 7) * 8 + (k & 7)


def tt_target(nc, r, j, col):
    """Steps 3-4 as tt_store restates them: column col of source node j's
    sums is meant for the sibling i in its slot qv; it lands at column
    k = qp r + cr of i's prepared operand (qp: j's slot among i's siblings)."""
    cj = j % nc
    qv, cr = divmod(col, r)
    ci = qv if qv < cj else qv + 1
    qp = cj if cj < ci else cj - 1
    return j - cj + ci, qp * r + cr


def replay_tc(g, NP, sms=152, seg=None):
    """Addresses of the TMA-fed tensor-core kernels (bf16 storage, NP
    right-hand-side columns): every V, U and D box start inside its map (x
    on 16 bytes; a box may run past the end, where the copy engine fills
    zeros for a load), every bulk copy of prepared x or t inside its region,
    every prepared-operand store and every T store inside its buffer, and
    the Step-2 reads of every node spanning accumulation segments (`seg`
    tiles from each range start; None: whole ranges) exactly on the partial
    slots the epilogue wrote."""
    bad = []
    tile, Np, s, G = g["tile"], g["Np"], g["s"], g["G"]
    KNP = 64                                    # rows of a prepared region
    xprep = Np * KNP
    tt_off, tt = {}, 0
    for l, L in g["lv"].items():
        tt_off[l] = tt
        L["srp64"] = (L["sr"] + 63) // 64 * 64
        tt += L["nodes"] * KNP * L["srp64"]
    # x prep stores: tile t, slot k < tile, row n < 64
    if (Np // tile - 1) * KNP * tile + prep_elem(63, tile - 1) >= xprep:
        bad.append("xprep store")
    # project: ranges of R tiles; per 64-slot chunk the x chunk and per
    # (level, 128-column block) one V box
    ntile = Np // tile
    R = -(-ntile // sms)
    written = {}
    for t in range(ntile):
        p0 = t * tile
        for kc in range(tile // 64):
            xo = t * KNP * tile + kc * 4096
            if xo + NP * 64 > xprep:
                bad.append(("x chunk", t, kc))
            for l, L in g["lv"].items():
                node = p0 // L["n"]
                x = p0 - node * L["n"] + kc * 64
                if not (0 <= x < L["n"] and (x * 2) % 16 == 0 and x + 64 <= L["n"]):
                    bad.append(("V box x", l, t))
                for cb in range(-(-L["sr"] // 128)):
                    y = node * L["sr"] + cb * 128
                    rows = min(128, L["sr"] - cb * 128)
                    if not (0 <= y and y + rows <= L["nodes"] * L["sr"]):
                        bad.append(("V box y", l, t, cb))
        # epilogue stores: node sum (whole node in the segment) or a partial
        # at the covered part's first tile
        tb, te = (t // R) * R, min((t // R) * R + R, ntile)
        F = seg or R
        sb = tb + (t - tb) // F * F
        se = min(sb + F, te)
        for l, L in g["lv"].items():
            tpn = max(L["n"] // tile, 1)
            node = p0 // L["n"]
            ns, ne = node * tpn, (node + 1) * tpn
            if ns >= sb and ne <= se:
                # a node sum goes to its targets' prepared operands
                for col in (0, L["sr"] - 1):
                    i, k = tt_target(s + 1, L["r"], node, col)
                    at = tt_off[l] + i * KNP * L["srp64"] + prep_elem(63, k)
                    if not (0 <= i < L["nodes"] and i // (s + 1) == node // (s + 1) and
                            tt_off[l] <= at < tt_off[l] + L["nodes"] * KNP * L["srp64"]):
                        bad.append(("t store (project)", l, t))
                continue
            else:
                pslot = max(ns, sb)
                written.setdefault((l, node), set()).add(pslot)
                idx = L["part"] + pslot * L["sr"] + L["sr"] - 1
                lo, hi = L["part"], L["part"] + ntile * L["sr"]
            if not (lo <= idx < hi) or idx >= g["T"]:
                bad.append(("T store", l, t))
    # Step 2: a spanning node reads its first tile and every segment start
    # inside it -- exactly the slots written above; the host lists the
    # spanning nodes from the segment starts (range starts, then F apart
    # inside a range), and that list must be exactly the nodes with reads
    F = seg or R
    for l, L in g["lv"].items():
        tpn = max(L["n"] // tile, 1)
        if tpn <= 1:
            continue
        listed, last = [], -1
        for c in range(-(-ntile // R)):
            for s0 in range(c * R + (F if c == 0 else 0), min((c + 1) * R, ntile), F):
                if s0 % tpn == 0:
                    continue
                j = s0 // tpn
                if j != last:
                    listed.append(j)
                    last = j
        if len(set(listed)) != len(listed):
            bad.append(("span list repeats", l))
        spanning = []
        for node in range(L["nodes"]):
            t0, t1 = node * tpn, (node + 1) * tpn
            inner = [t for t in range(t0 + 1, t1) if (t % R) % F == 0]
            reads = {t0, *inner} if inner else set()
            if reads != written.get((l, node), set()):
                bad.append(("step-2 reads", l, node))
            if inner:
                spanning.append(node)
        if sorted(listed) != spanning:
            bad.append(("span list", l))
    # Steps 3-4 routing: over a level, (source, column) -> (target, column)
    # is one to one onto every target's columns k < s r (the padding columns
    # stay untouched), inside the sibling group, and every store lands in
    # the level's region
    for l, L in g["lv"].items():
        hit = {}
        for j in range(L["nodes"]):
            for col in range(L["sr"]):
                i, k = tt_target(s + 1, L["r"], j, col)
                hit[(i, k)] = hit.get((i, k), 0) + 1
                if i // (s + 1) != j // (s + 1) or i == j or not (0 <= k < L["sr"]):
                    bad.append(("t routing", l, j, col))
        if set(hit) != {(i, k) for i in range(L["nodes"]) for k in range(L["sr"])} or \
                any(v != 1 for v in hit.values()):
            bad.append(("t routing not one to one", l))
        last = tt_off[l] + (L["nodes"] - 1) * KNP * L["srp64"] + prep_elem(63, L["sr"] - 1)
        if last >= tt_off[l] + L["nodes"] * KNP * L["srp64"]:
            bad.append(("t store", l))
    # expand: 128-slot tiles; per stage two A boxes (slots x, x + 64) and one B chunk
    for t in range(Np // 128):
        e0 = t * 128
        grp = e0 // G
        for c0 in range(0, G, 64):
            x = e0 - grp * G
            if not (0 <= x and x + 128 <= G) or grp * G + c0 >= (Np // G) * G:
                bad.append(("D box", t))
            slot = grp * G + c0
            tp = slot // tile
            at0 = tp * KNP * tile + ((slot - tp * tile) >> 6) * 4096
            if at0 + NP * 64 > xprep:
                bad.append(("x chunk (expand)", t))
        for l, L in g["lv"].items():
            node = e0 // L["n"]
            x = e0 - node * L["n"]
            srp = (L["sr"] + 15) // 16 * 16
            for c0 in range(0, srp, 64):
                y = node * L["sr"] + c0
                if not (0 <= x and x + 128 <= L["n"]) or not (0 <= y < L["nodes"] * L["sr"]):
                    bad.append(("U box", l, t, c0))
                at0 = tt_off[l] + node * KNP * L["srp64"] + (c0 >> 6) * 4096
                if at0 + NP * 64 > tt_off[l] + L["nodes"] * KNP * L["srp64"]:
                    bad.append(("t chunk", l, t, c0))
    return bad


@pytest.mark.parametrize("d,n,r,NP", [(3, 64, 32, 32), (2, 1024, 16, 64), (2, 128, 16, 64),
                                      (3, 16, 8, 32), (2, 256, 4, 16)])
@pytest.mark.parametrize("seg", [None, 4])
def test_tensor_core_addressing_in_bounds(hm, d, n, r, NP, seg):
    opts = hm.hmat_default_opts(device=-1, method=2, seed=5, prec=2)
    h = hm.hmat_build(w.grid_points(n, d), 2, 64, r, 0.0, opts)
    try:
        g = geometry(hm.hmat_info(h))
    finally:
        hm.hmat_destroy(h)
    assert g["G"] % 128 == 0 and g["Np"] % 128 == 0 and g["G"] % g["tile"] == 0
    assert replay_tc(g, NP, seg=seg) == []


def test_replays_catch_planted_mistakes(hm):
    """The replays are not vacuous: a partial-sum buffer one entry short, or
    a level whose map is one node short, is reported."""
    opts = hm.hmat_default_opts(device=-1, method=2, seed=5, prec=1)
    h = hm.hmat_build(w.grid_points(64, 2), 2, 64, 4, 0.0, opts)
    try:
        info = hm.hmat_info(h)
    finally:
        hm.hmat_destroy(h)
    g = geometry(info)
    g["T"] -= 1
    assert any(b[0] == "T store" for b in replay(g, 4))
    g = geometry(info)
    g["lv"][1]["nodes"] -= 1
    assert any(b[0] in ("V box y", "U box y", "T read") for b in replay(g, 4))
    assert any(b[0] in ("V box y", "U box") for b in replay_tc(g, 32))
