"""Host-side models of the sort's device logic, checked on the CPU against the oracle's bin/sort
(App. C.2) and against plain stable sorts.  No kernel runs here: the models restate, step by
step, what the kernels of the tile binning do, so that a slip in the window arithmetic or in
the block/warp prefix structure shows up without a GPU.

- ``emit_window`` is the warp-level slot generation: pair j owns slots [offsets[j],
  offsets[j] + count_j) and covers a rectangle of tiles; the pairs starting inside a window of
  32 slots are found from one OR of their start bits, each slot takes its pair's data from the
  lane that loaded it, and splits its index in the rectangle into row and column with a float
  quotient corrected by integer steps.
- ``rank_pass`` is one stable counting pass over blocks of 16 warp segments: per-block digit
  counts, digit-major exclusive scan, per-warp counters turned into prefixes, and ranking of 32
  items at a time by lane among equal digits."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2409_06765_gb300 import _lib, synth


def _support_span(m, r):
    m2 = np.clip(np.float32(2.0) * np.float32(m), np.float32(-268435456.0), np.float32(268435456.0))
    a = int(np.ceil(m2)) - 2 * r
    b = int(np.floor(m2)) + 2 * r
    return a >> 1, (b - 1) >> 1


def _pairs_in_depth_order(means2d, depths, radii, widths, heights, t):
    """Visible pairs in (depth bits, flat index) order with their tile rectangles, packed as the
    count kernel packs them: (global first tile, width | tiles per row << 16)."""
    C, N = depths.shape
    tiles_x = [-(-w // t) for w in widths]
    tile_off = np.concatenate([[0], np.cumsum([tiles_x[c] * -(-heights[c] // t) for c in range(C)])])
    keys = depths.reshape(-1).view(np.uint32).astype(np.int64)
    order, counts, rects = [], [], []
    for i in np.argsort(keys, kind="stable"):
        c, n = divmod(int(i), N)
        r = int(radii[c, n])
        if r <= 0:
            continue
        x0, x1 = _support_span(means2d[c, n, 0], r)
        y0, y1 = _support_span(means2d[c, n, 1], r)
        x0, y0, x1, y1 = max(x0, 0), max(y0, 0), min(x1, widths[c] - 1), min(y1, heights[c] - 1)
        if x0 > x1 or y0 > y1:
            continue
        tx0, tx1, ty0, ty1 = x0 // t, x1 // t, y0 // t, y1 // t
        order.append(int(i))
        counts.append((tx1 - tx0 + 1) * (ty1 - ty0 + 1))
        rects.append((int(tile_off[c]) + ty0 * tiles_x[c] + tx0, (tx1 - tx0 + 1) | (tiles_x[c] << 16)))
    return np.array(order, np.int64), np.array(counts, np.int64), np.array(rects, np.int64).reshape(-1, 2)


def _f32_quotient(k, w, rcp_ulps=0):
    """k / w as the emission computes it: a float32 estimate of (k + 0.5) / w from a reciprocal
    (``rcp_ulps`` ulps away from the correctly rounded one, as the hardware approximation may
    be), truncated, then one correction step of -1, 0 or +1."""
    r32 = np.float32(np.float32(1.0) / np.float32(w))
    for _ in range(abs(rcp_ulps)):
        r32 = np.nextafter(r32, np.float32(np.inf if rcp_ulps > 0 else -np.inf), dtype=np.float32)
    q = int(np.float32(np.float32(np.float32(k) + np.float32(0.5)) * r32))
    r = k - q * w
    adj = -1 if r < 0 else (1 if r >= w else 0)
    return q + adj, r - adj * w


def emit_window(offsets, rects, order, win_start, w0, n_slots):
    """Tiles and values of slots [w0, w0 + 32), as the 32 lanes of a warp compute them."""
    npairs = len(offsets)
    pc = win_start[w0 // 32]
    off = [offsets[pc + l] if pc + l < npairs else 1 << 62 for l in range(32)]
    starts = 0
    for lane in range(1, 32):
        st = off[lane] - w0
        if 0 <= st < 32:
            starts |= 1 << st
    out = []
    for lane in range(32):
        jl = bin(starts & ((1 << (lane + 1)) - 1)).count("1")
        q = w0 + lane
        if q >= n_slots:
            out.append(None)
            continue
        j = pc + jl
        base, wt = rects[j]
        w, tx = wt & 0xFFFF, wt >> 16
        ky, kx = _f32_quotient(int(q - off[jl]), w)
        out.append((base + ky * tx + kx, int(order[j]), jl))
    return out


def pair_loop_ranks(window, counters):
    """Ranks of a window's slots as the place kernel assigns them: the window's pairs one after
    the other, each lane of the current pair reading and bumping its tile's counter."""
    ranks = [None] * 32
    npair = 1 + max((s[2] for s in window if s is not None), default=0)
    for p in range(npair):
        for lane, s in enumerate(window):
            if s is not None and s[2] == p:
                ranks[lane] = counters.get(s[0], 0)
                counters[s[0]] = ranks[lane] + 1
    return ranks


def _window_starts(offsets, counts, n_slots):
    win = np.full((n_slots + 31) // 32 + 1, -1, np.int64)
    for j, (o, c) in enumerate(zip(offsets, counts)):
        end = min(o + c, n_slots)
        w = (o + 31) // 32
        while 32 * w < end:
            win[w] = j
            w += 1
    return win


def _scene_lists(seed, C, t, sizes):
    sc = synth.clustered_scene(1500, seed, sh_degree=0, log_scale_mu=-2.6)
    cams = synth.sphere_cameras(seed, sizes[:C])
    sp = [oracle.project(sc, cam) for cam in cams]
    m = np.stack([p["means2d"] for p in sp]).astype(np.float32)
    d = np.stack([p["depths"] for p in sp]).astype(np.float32)
    r = np.stack([p["radii"] for p in sp])
    return m, d, r, [c.width for c in cams], [c.height for c in cams]


@pytest.mark.parametrize("t", [8, 16, 32])
def test_emission_windows_regenerate_the_oracles_slots(t):
    m, d, r, W, H = _scene_lists(4, 3, t, [(97, 61), (160, 90), (33, 200)])
    order, counts, rects = _pairs_in_depth_order(m, d, r, W, H, t)
    offsets = np.concatenate([[0], np.cumsum(counts)[:-1]])
    K = int(counts.sum())
    win = _window_starts(offsets, counts, K)
    slots, counters, ranks = [], {}, []
    for w0 in range(0, K, 32):
        win_slots = emit_window(offsets, rects, order, win, w0, K)
        for p in set(s[2] for s in win_slots if s is not None):  # a pair's slots are distinct tiles
            tl = [s[0] for s in win_slots if s is not None and s[2] == p]
            assert len(tl) == len(set(tl))
        ranks += [r for r in pair_loop_ranks(win_slots, counters) if r is not None]
        slots += [s for s in win_slots if s is not None]
    tiles = np.array([s[0] for s in slots])
    vals = np.array([s[1] for s in slots])
    # the per-pair ranking numbers each tile's slots 0, 1, 2, ... in slot order
    for tl in np.unique(tiles):
        np.testing.assert_array_equal(np.array(ranks)[tiles == tl], np.arange((tiles == tl).sum()))
    # the slots in depth order, stably sorted by tile, are the oracle's list
    keys_r, vals_r, _ = oracle.bin_sort(m, d, r, W, H, t)
    o = np.argsort(tiles, kind="stable")
    np.testing.assert_array_equal(vals[o], vals_r)
    np.testing.assert_array_equal(tiles[o], (keys_r >> np.uint64(32)).astype(np.int64))


def test_window_start_bits_from_the_pair_offsets_equal_the_warp_or():
    """The offsets kernel sets bit (off & 31) of window off >> 5 for every pair that starts
    inside a window; that is the OR of the start bits the lanes of the window would compute."""
    m, d, r, W, H = _scene_lists(6, 2, 16, [(120, 90), (64, 200)])
    order, counts, rects = _pairs_in_depth_order(m, d, r, W, H, 16)
    offsets = np.concatenate([[0], np.cumsum(counts)[:-1]])
    for n_slots in (int(counts.sum()), int(counts.sum()) // 3):
        win = _window_starts(offsets, counts, n_slots)
        bits = np.zeros(len(win), np.int64)
        for o in offsets:
            if o < n_slots and o & 31:
                bits[o >> 5] |= 1 << (o & 31)
        for w0 in range(0, n_slots, 32):
            pc = win[w0 // 32]
            ref = 0
            for lane in range(1, 32):
                if pc + lane < len(offsets) and 0 <= offsets[pc + lane] - w0 < 32:
                    ref |= 1 << int(offsets[pc + lane] - w0)
            assert bits[w0 // 32] == ref


def test_emission_windows_with_single_slot_pairs_and_a_capacity_cut():
    # 70 pairs of one slot, then a pair of 5 x 3 tiles, then single slots again; windows where
    # all 32 lanes start a new pair, and a slot limit that ends inside a pair
    counts = np.array([1] * 70 + [15] + [1] * 40, np.int64)
    rects = np.array([(k, 1 | (9 << 16)) for k in range(70)] + [(100, 5 | (9 << 16))] +
                     [(200 + k, 1 | (9 << 16)) for k in range(40)], np.int64)
    order = np.arange(len(counts)) * 7
    offsets = np.concatenate([[0], np.cumsum(counts)[:-1]])
    for n_slots in (int(counts.sum()), 77, 96):
        win = _window_starts(offsets, counts, n_slots)
        got = []
        for w0 in range(0, n_slots, 32):
            got += [s[:2] for s in emit_window(offsets, rects, order, win, w0, n_slots) if s is not None]
        want = []
        for j, c in enumerate(counts):
            base, wt = rects[j]
            w, tx = wt & 0xFFFF, wt >> 16
            want += [(int(base + (k // w) * tx + k % w), int(order[j])) for k in range(c)]
        assert got == want[:n_slots]


def test_float_quotient_with_one_correction_step_is_exact():
    """Slot k of a rectangle of width w <= 4096 tiles and at most 4096 rows (a camera of up to
    32768 pixels a side at 8-pixel tiles): one correction step after the float estimate gives
    the exact row and column, also with a reciprocal off by a couple of ulps."""
    rng = np.random.default_rng(3)
    w = rng.integers(1, 4097, 40000)
    k = (rng.random(40000) * w * rng.integers(1, 4097, 40000)).astype(np.int64)
    for kk, ww in zip(k, w):
        for ulps in (-2, 0, 2):
            assert _f32_quotient(int(kk), int(ww), ulps) == divmod(int(kk), int(ww))
    for ww in (1, 3, 7, 60, 4096):  # the extremes of each width: first and last slot of 4096 rows
        for kk in (0, ww - 1, ww, 4096 * ww - 1):
            assert _f32_quotient(kk, ww, 2) == divmod(kk, ww)


def rank_pass(keys, vals, shift, bits, seg, warps=16, drop=None):
    """One stable counting pass as the histogram, scan and rank kernels compute it."""
    n = len(keys)
    block = warps * seg
    nd = 1 << bits
    digit = (keys >> shift) & (nd - 1)
    keep = np.ones(n, bool) if drop is None else keys != drop
    nb = (n + block - 1) // block
    hist = np.zeros((nd, max(nb, 1)), np.int64)
    for b in range(nb):
        sl = slice(b * block, min((b + 1) * block, n))
        hist[:, b] = np.bincount(digit[sl][keep[sl]], minlength=nd)
    rowsum = hist.sum(1)
    start = np.concatenate([[0], np.cumsum(rowsum)[:-1]])[:, None] + \
        np.concatenate([np.zeros((nd, 1), np.int64), np.cumsum(hist, 1)[:, :-1]], 1)
    out_k = np.full(int(keep.sum()), -1, np.int64)
    out_v = np.full(int(keep.sum()), -1, np.int64)
    for b in range(nb):
        cnt = np.zeros((warps, nd), np.int64)
        for w in range(warps):
            s0, s1 = b * block + w * seg, min(b * block + (w + 1) * seg, n)
            for q in range(s0, s1):
                if keep[q]:
                    cnt[w, digit[q]] += 1
        pre = np.concatenate([np.zeros((1, nd), np.int64), np.cumsum(cnt, 0)[:-1]], 0)
        for w in range(warps):
            s0, s1 = b * block + w * seg, min(b * block + (w + 1) * seg, n)
            for w0 in range(s0, s1, 32):
                lanes = [q for q in range(w0, min(w0 + 32, s1)) if keep[q]]
                for q in lanes:  # rank among the lanes of this step with the same digit
                    peers_before = sum(1 for p in lanes if p < q and digit[p] == digit[q])
                    pos = start[digit[q], b] + pre[w, digit[q]] + peers_before
                    out_k[pos], out_v[pos] = keys[q], vals[q]
                for dd in set(digit[q] for q in lanes):
                    pre[w, dd] += sum(1 for q in lanes if digit[q] == dd)
    return out_k, out_v


@pytest.mark.parametrize("bits,seg,n", [(11, 32, 3000), (11, 64, 2500), (4, 32, 1100), (10, 96, 2049)])
def test_counting_pass_model_is_a_stable_sort(bits, seg, n):
    rng = np.random.default_rng(bits + seg)
    keys = rng.integers(0, 1 << 22, n)
    keys[::5] = keys[3]  # many equal digits
    vals = np.arange(n) * 3
    out_k, out_v = rank_pass(keys, vals, 3, bits, seg)
    o = np.argsort((keys >> 3) & ((1 << bits) - 1), kind="stable")
    np.testing.assert_array_equal(out_k, keys[o])
    np.testing.assert_array_equal(out_v, vals[o])


def test_three_passes_dropping_invisible_keys_give_the_depth_order():
    rng = np.random.default_rng(5)
    n = 2600
    depth = rng.choice(rng.uniform(0.3, 9.0, 300), n).astype(np.float32)
    keys = depth.view(np.uint32).astype(np.int64)
    keys[rng.random(n) < 0.3] = 0xFFFFFFFF  # pairs without tiles
    vals = np.arange(n)
    k, v = keys, vals
    for i, (shift, bits) in enumerate(((0, 11), (11, 11), (22, 10))):
        k, v = rank_pass(k, v, shift, bits, 32, drop=0xFFFFFFFF if i == 0 else None)
    vis = keys != 0xFFFFFFFF
    o = np.lexsort((vals[vis], keys[vis]))
    np.testing.assert_array_equal(v, vals[vis][o])


def test_intersection_capacity_above_the_int32_limit_is_a_capacity_error():
    lib = _lib.load()
    cams = _lib.CameraArray([synth.make_camera(32, 32, (0, 0, 4))])
    p = _lib.make_params()
    fake, null = ctypes.c_void_p(256), ctypes.c_void_p(None)
    big = _lib.GS_MAX_INTERSECTIONS + 1
    assert lib.gs_tile_bin_sort_workspace(cams.ptr, 1, 10, ctypes.byref(p), big) == -1
    st = lib.gs_tile_bin_sort(cams.ptr, 1, 10, ctypes.byref(p), fake, fake, fake, big, null, fake, fake, fake, fake,
                              1 << 40, null)
    assert st == _lib.GS_ERR_CAPACITY and b"GS_MAX_INTERSECTIONS" in lib.gs_last_error()
    assert lib.gs_tile_bin_sort_noalloc(cams.ptr, 1, 10, ctypes.byref(p), fake, fake, fake, big, null, fake, fake,
                                        fake, null) == _lib.GS_ERR_CAPACITY
    with pytest.raises(_lib.GsError) as ei:
        _lib.gs_tile_bin_sort_workspace(cams, 10, p, big)
    assert ei.value.status == _lib.GS_ERR_CAPACITY
    # the limit itself is a valid capacity
    assert lib.gs_tile_bin_sort_workspace(cams.ptr, 1, 10, ctypes.byref(p), _lib.GS_MAX_INTERSECTIONS) > 0


def test_single_pass_workspace_holds_nothing_of_the_list_size():
    """Up to 2048 tiles the sort keeps no K-sized arrays: the workspace grows by under one byte
    per slot of capacity (block counts and window starts); past 2048 tiles it holds (tile,
    value) arrays and a second value array, 12 bytes per slot."""
    p = _lib.make_params(tile=32)
    one = _lib.CameraArray([synth.make_camera(1920, 1080, (0, 0, 4))])  # 2040 tiles
    a = _lib.gs_tile_bin_sort_workspace(one, 1000, p, 1_000_000)
    b = _lib.gs_tile_bin_sort_workspace(one, 1000, p, 9_000_000)
    assert 0 < (b - a) / 8_000_000 < 1.0
    many = _lib.CameraArray([synth.make_camera(1920, 1080, (0, 0, 4))] * 2)  # 4080 tiles
    a = _lib.gs_tile_bin_sort_workspace(many, 1000, p, 1_000_000)
    b = _lib.gs_tile_bin_sort_workspace(many, 1000, p, 9_000_000)
    assert (b - a) / 8_000_000 >= 12.0
