"""The work schedule of the wavefront step (k_wave), restated on the host:
items k = g * tp + T (group g = 0 .. nz + lag - 1, tile T of 32 x by nodes
of a plane, tp tiles per plane) sum plane (g - 1) mod nz of their tile and
collide plane g - lag of it once the 27 tiles around it in planes
q - 1 .. q + 1 are summed.  Checked here for the tile shapes and lags the
library offers and for ragged and degenerate lattices:
  - every (plane, tile) is summed once and collided once, after its own sum;
  - flag indices fall inside the workspace's flag words;
  - every tile a node's stencil reaches is one of the 27 whose flags are
    polled (periodic wrap included);
  - a collision waits only on items of earlier groups when lag >= 3, and a
    greedy run of blocks that take tickets in order finishes (no deadlock),
    while lag = 2 can wait on a later item;
  - several lattices in one launch (items numbered group-major across the
    batch, the segment arithmetic the launch uses checked against a plain
    enumeration) keep every wait inside the waiting item's own lattice and on
    a smaller ticket, and a greedy run of blocks finishes."""
import pytest

BY_OF_SHAPE = {1: 4, 2: 2, 3: 8}
SIZES = [(7, 4, 5), (33, 9, 3), (64, 20, 17), (40, 1, 2), (256, 12, 1), (32, 8, 9),
         (100, 17, 6), (1, 3, 4), (96, 40, 12)]


def flag_words(nx, ny, nz):
    """Flags the workspace holds (one per x-tile)."""
    return nz * ny * ((nx + 31) // 32)


def schedule(nx, ny, nz, by, lag):
    ntx = (nx + 31) // 32
    nty = (ny + by - 1) // by
    tp = ntx * nty
    items = []
    for k in range((nz + lag) * tp):
        grp, T = divmod(k, tp)
        tx, ty = T % ntx, T // ntx
        q = grp - lag
        zd = nz - 1 if grp == 0 else grp - 1
        waits = []
        if q >= 0:
            for l in range(27):
                dx, dy, dz = l % 3 - 1, (l // 3) % 3 - 1, l // 9 - 1
                zz, yy, xx = (q + dz) % nz, (ty + dy) % nty, (tx + dx) % ntx
                waits.append(zz * tp + yy * ntx + xx)
        items.append({"grp": grp, "T": T, "sum": (zd, T) if grp < nz else None,
                      "collide": (q, T) if q >= 0 else None, "waits": waits,
                      "flag": zd * tp + T if grp < nz else None})
    return items, tp, ntx, nty


@pytest.mark.parametrize("shape", sorted(BY_OF_SHAPE))
@pytest.mark.parametrize("lag", [3, 4, 5, 7])
def test_each_tile_summed_and_collided_once(shape, lag):
    by = BY_OF_SHAPE[shape]
    for nx, ny, nz in SIZES:
        items, tp, ntx, nty = schedule(nx, ny, nz, by, lag)
        summed, collided = {}, {}
        for k, it in enumerate(items):
            if it["sum"] is not None:
                assert it["sum"] not in summed
                summed[it["sum"]] = it["grp"]
                assert 0 <= it["flag"] < nz * tp <= flag_words(nx, ny, nz)
            if it["collide"] is not None:
                assert it["collide"] not in collided
                collided[it["collide"]] = it["grp"]
            for fi in it["waits"]:
                assert 0 <= fi < nz * tp
        assert len(summed) == len(collided) == nz * tp
        for key, g in collided.items():
            assert summed[key] < g          # a tile is summed before it is collided


@pytest.mark.parametrize("by", [2, 4, 8])
def test_stencil_stays_in_the_polled_tiles(by):
    for nx, ny, nz in SIZES:
        ntx, nty = (nx + 31) // 32, (ny + by - 1) // by
        for y in range(ny):
            for dy in (-1, 1):
                assert ((y + dy) % ny) // by in {(y // by + d) % nty for d in (-1, 0, 1)}
        for x in range(nx):
            for dx in (-1, 1):
                assert ((x + dx) % nx) // 32 in {(x // 32 + d) % ntx for d in (-1, 0, 1)}


def _flag_group(items, tp):
    """Group of the item that sets each flag."""
    return {it["flag"]: it["grp"] for it in items if it["flag"] is not None}


@pytest.mark.parametrize("lag", [3, 4, 6])
def test_waits_point_to_earlier_groups(lag):
    for nx, ny, nz in SIZES:
        for by in (2, 4, 8):
            items, tp, _, _ = schedule(nx, ny, nz, by, lag)
            setter = _flag_group(items, tp)
            for it in items:
                for fi in it["waits"]:
                    assert setter[fi] < it["grp"]


def _greedy_run(items, blocks):
    """Blocks take tickets in order, one item at a time; an item finishes
    when the flags it waits on are set, then sets its own.  Returns True if
    every item finishes."""
    done_flags, nxt, holding = set(), 0, [None] * blocks
    finished = 0
    while True:
        progress = False
        for b in range(blocks):
            if holding[b] is None and nxt < len(items):
                holding[b] = nxt
                nxt += 1
                progress = True
            k = holding[b]
            if k is not None and all(f in done_flags for f in items[k]["waits"]):
                if items[k]["flag"] is not None:
                    done_flags.add(items[k]["flag"])
                holding[b] = None
                finished += 1
                progress = True
        if finished == len(items):
            return True
        if not progress:
            return False


@pytest.mark.parametrize("blocks", [1, 3, 64])
def test_ticket_order_finishes(blocks):
    for nx, ny, nz in [(64, 20, 17), (33, 9, 3), (7, 4, 5), (40, 1, 2)]:
        items, _, _, _ = schedule(nx, ny, nz, 2, 4)
        assert _greedy_run(items, blocks)


def test_lag_two_can_wait_on_a_later_item():
    """Why the library rejects lag < 3: with lag 2 some collision waits on a
    tile summed in its own group."""
    items, tp, _, _ = schedule(64, 20, 17, 2, 2)
    setter = _flag_group(items, tp)
    assert any(setter[fi] >= it["grp"] for it in items for fi in it["waits"])


def _batch_order(sizes, by, lag, budget=float("inf"), node_bytes=152):
    """Lattices by group count, most first (stable), cut into sets whose
    planes in flight ((lag + 2) planes of x-tile-padded rows) fit `budget`
    bytes together (a lattice alone may exceed it); tiles per plane and
    group counts."""
    tps = [((nx + 31) // 32) * ((ny + by - 1) // by) for nx, ny, nz in sizes]
    groups = [nz + lag for nx, ny, nz in sizes]
    order = sorted(range(len(sizes)), key=lambda r: -groups[r])
    sets, cur, used = [], [], 0.0
    for r in order:
        nx, ny, nz = sizes[r]
        b = (lag + 2) * ((nx + 31) // 32) * 32 * ny * node_bytes
        if cur and used + b > budget:
            sets.append(cur)
            cur, used = [], 0.0
        cur.append(r)
        used += b
    sets.append(cur)
    return sets, tps, groups


def _segment_lookup(sizes, by, lag, budget=float("inf")):
    """ticket -> (lattice, item of that lattice) by the launch's segment
    arithmetic: inside each set, groups [G_m, G_(m-1)) hold the set's m
    lattices with most groups, their tiles per plane summed per group."""
    sets, tps, groups = _batch_order(sizes, by, lag, budget)
    order = [r for st in sets for r in st]
    tsum = [0]
    for r in order:
        tsum.append(tsum[-1] + tps[r])
    segs, first, lb = [], 0, 0
    for st in sets:
        g0 = 0
        for m in range(len(st), 0, -1):
            gend = groups[order[lb + m - 1]]
            if gend <= g0:
                continue
            segs.append((first, g0, lb, m))
            first += (gend - g0) * (tsum[lb + m] - tsum[lb])
            g0 = gend
        lb += len(st)

    def lookup(k):
        s = max(i for i, sg in enumerate(segs) if sg[0] <= k)
        f0, gs, lb, m = segs[s]
        gg, rem = divmod(k - f0, tsum[lb + m] - tsum[lb])
        rem += tsum[lb]
        l = max(i for i in range(lb, lb + m) if tsum[i] <= rem)
        r = order[l]
        return r, (gs + gg) * tps[r] + rem - tsum[l]
    return lookup, first


def _batch_schedule(sizes, by, lag, budget=float("inf")):
    """Items of several lattices in one launch: set after set, group-major
    inside a set (group g of every lattice of the set that has one, in
    order of group count, before group g + 1).  Each item's lattice, and
    its waits as (lattice, flag)."""
    sets, tps, groups = _batch_order(sizes, by, lag, budget)
    per = [schedule(nx, ny, nz, by, lag)[0] for nx, ny, nz in sizes]
    items = []
    for st in sets:
        for g in range(max(groups[r] for r in st)):
            for r in st:
                if g >= groups[r]:
                    continue
                for T in range(tps[r]):
                    it = per[r][g * tps[r] + T]
                    items.append({"r": r, "local": g * tps[r] + T, "grp": g,
                                  "waits": [(r, f) for f in it["waits"]],
                                  "flag": (r, it["flag"]) if it["flag"] is not None else None})
    return items


BUDGETS = [float("inf"), 0.0, 2.0e6]


@pytest.mark.parametrize("by", [2, 4])
@pytest.mark.parametrize("budget", BUDGETS)
def test_segment_arithmetic_numbers_the_batch(by, budget):
    for sizes in ([(40, 9, 5), (7, 4, 3), (64, 20, 6), (33, 1, 2)],
                  [(32, 32, 32), (64, 64, 64), (33, 7, 64), (96, 5, 1)],
                  [(16, 3, 9)], [(8, 8, 4), (8, 8, 4), (40, 2, 4)]):
        items = _batch_schedule(sizes, by, 4, budget)
        lookup, total = _segment_lookup(sizes, by, 4, budget)
        assert total == len(items) == sum((nz + 4) * ((nx + 31) // 32) * ((ny + by - 1) // by)
                                           for nx, ny, nz in sizes)
        assert [lookup(k) for k in range(total)] == [(it["r"], it["local"]) for it in items]
        assert len({(it["r"], it["local"]) for it in items}) == total


def test_sets_follow_the_budget():
    sizes = [(32, 32, 32), (64, 64, 64), (33, 7, 64), (96, 5, 1)]
    assert len(_batch_order(sizes, 2, 4)[0]) == 1
    assert _batch_order(sizes, 2, 4, 0.0)[0] == [[1], [2], [0], [3]]
    # 64^2 x 6 planes x 152 B = 3.7 MB: alone in a 2 MB set, the rest share
    assert _batch_order(sizes, 2, 4, 2.0e6)[0] == [[1], [2, 0, 3]]


@pytest.mark.parametrize("by", [2, 4])
@pytest.mark.parametrize("budget", BUDGETS)
def test_batched_items_wait_inside_their_lattice(by, budget):
    sizes = [(40, 9, 5), (7, 4, 3), (64, 20, 6), (33, 1, 2)]
    items = _batch_schedule(sizes, by, 4, budget)
    setter = {it["flag"]: k for k, it in enumerate(items) if it["flag"] is not None}
    for k, it in enumerate(items):
        for wflag in it["waits"]:
            assert wflag[0] == it["r"]
            assert setter[wflag] < k
    for blocks in (1, 5, 64):
        done, nxt, holding, finished = set(), 0, [None] * blocks, 0
        while finished < len(items):
            progress = False
            for b in range(blocks):
                if holding[b] is None and nxt < len(items):
                    holding[b], nxt, progress = nxt, nxt + 1, True
                k = holding[b]
                if k is not None and all(w in done for w in items[k]["waits"]):
                    if items[k]["flag"] is not None:
                        done.add(items[k]["flag"])
                    holding[b], finished, progress = None, finished + 1, True
            assert progress
