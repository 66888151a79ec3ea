"""C-ABI checks that need no GPU: the library loads, exports every entry point
that include/fw.h declares, rejects bad arguments on the host before touching
CUDA, and its persistent task queue is a valid topological order."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fw.h")


@pytest.fixture(scope="module")
def fw():
    import paper_2403_18619_gb300 as fw
    from paper_2403_18619_gb300 import build
    if not os.path.exists(fw.LIB_PATH):
        build.build()
    fw.load()
    return fw


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fw_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(fw):
    names = declared_functions()
    assert len(names) >= 15
    lib = fw.load()
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", fw.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (fw_[a-z_0-9]+)", out))
    assert set(names) <= exported


def test_status_strings_and_defaults(fw):
    lib = fw.load()
    for code in range(7):
        assert lib.fw_status_string(code)
    o = fw.Options.default()
    assert o.bs == 0 and o.packed_keys == 1 and o.debug_skip_release == -1 and o.lookahead == -1
    assert o.tile_tma == 1


def test_options_mirror_matches_header(fw, tmp_path):
    """The binding's ctypes mirror of fw_options has the header's size and
    field offsets (a C program compiled against include/fw.h prints them)."""
    fields = [f for f, _ in fw.Options._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"fw.h\"\n"
                   "int main(void) {\n  printf(\"%zu\\n\", sizeof(fw_options));\n" +
                   "".join("  printf(\"%%zu\\n\", offsetof(fw_options, %s));\n" % f
                           for f in fields) + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got[0] == ctypes.sizeof(fw.Options)
    assert got[1:] == [getattr(fw.Options, f).offset for f in fields]


def test_host_argument_checks(fw):
    lib = fw.load()
    good = 0x10000  # never dereferenced: every call below fails its host-side checks
    I32 = fw.FW_I32
    assert lib.fw_solve(None, good + 4096, 8, 8, I32, None) == 1
    assert lib.fw_solve(good, good + 4096, 0, 8, I32, None) == 1
    assert lib.fw_solve(good, good + 4096, 9, 8, I32, None) == 1       # ld < n
    assert lib.fw_solve(good, good + 4096, 6, 6, I32, None) == 1       # ld % 4 != 0
    assert lib.fw_solve(good + 4, good + 4096, 8, 8, I32, None) == 1   # misaligned
    assert lib.fw_solve(good, good, 8, 8, I32, None) == 1              # aliasing
    assert lib.fw_solve(good, good + 4096, 8, 8, 7, None) == 1         # dtype
    bad = fw.Options.default(bs=48)
    assert lib.fw_solve_ex(good, good + 4096, 8, 8, I32, ctypes.byref(bad), None) == 1
    bad = fw.Options.default(driver=9)
    assert lib.fw_solve_ex(good, good + 4096, 8, 8, I32, ctypes.byref(bad), None) == 1
    bad = fw.Options.default(tile_tma=2)
    assert lib.fw_solve_ex(good, good + 4096, 8, 8, I32, ctypes.byref(bad), None) == 1
    assert lib.fw_solve_host(None, None, 8, 8, I32, None, None) == 1
    assert lib.fw_queue_tasks(0, 0, 0, 0, None) == 1
    assert lib.fw_verify_certificate(None, None, None, 8, 8, None, None) == 1


def _update_task(t):
    typ, r, i, j = t
    return (r, i, j)


@pytest.mark.parametrize("R,look", [(R, look) for R in (1, 2, 3, 4, 7, 12)
                                    for look in (0, 5, 10 ** 6)] +
                         [(32, "auto"), (24, "auto"), (40, "auto")])
def test_queue_is_complete_and_topological(fw, R, look):
    if look == "auto":
        # the lookahead a BS = 128 solve with R rounds gets on 152 SMs
        look = fw.fw_solve_plan(R * 128, fw.Options.default(bs=128), sms=152)["lookahead"]
    q = fw.fw_queue_tasks(R, look)
    assert q.shape == (R ** 3, 4)
    pos = {}
    for idx, (typ, r, i, j) in enumerate(q.tolist()):
        key = (r, i, j)
        assert key not in pos, "tile updated twice in one round"
        pos[key] = idx
        if i == r and j == r:
            assert typ == 0
        elif i == r:
            assert typ == 1
        elif j == r:
            assert typ == 2
        else:
            assert typ == 3
    assert len(pos) == R ** 3
    rounds_p2 = {}
    rounds_p3 = {}
    for idx, (typ, r, i, j) in enumerate(q.tolist()):
        if typ in (1, 2):
            rounds_p2.setdefault(r, []).append(idx)
        if typ == 3:
            rounds_p3.setdefault(r, []).append(idx)
    for idx, (typ, r, i, j) in enumerate(q.tolist()):
        deps = []
        if r >= 1:
            deps.append(pos[(r - 1, i, j)])        # the tile's own previous round
        if typ in (1, 2):
            deps.append(pos[(r, r, r)])            # the closed pivot
        if typ == 3:
            deps.append(pos[(r, i, r)])            # column panel tile of its row
            deps.append(pos[(r, r, j)])            # row panel tile of its column
        if typ == 0 and r >= 2:
            deps += rounds_p2.get(r - 2, [])       # pivot snapshot slot reuse
        if typ in (1, 2) and r >= 2:
            deps += rounds_p3.get(r - 2, [])       # panel snapshot slot reuse
        for d in deps:
            assert d < idx, (q[idx].tolist(), q[d].tolist())


def _check_order(q, pos):
    """Every dependency of the persistent engine precedes its task: q holds one
    graph's queue rows (type, round, tile row, tile column) by task index, pos
    the claim position of each task index.  Besides the queue's own rules, the
    task of tile (r+1, r+1) in round r runs the pivot of round r+1 too, so it
    also waits for that pivot's snapshot slot (the panels of round r-1) and
    precedes round r+1's panels."""
    at = {}
    p2, p3 = {}, {}
    for t, (typ, r, i, j) in enumerate(q.tolist()):
        at[(r, i, j)] = pos[t]
        if typ in (1, 2):
            p2.setdefault(r, []).append(pos[t])
        if typ == 3:
            p3.setdefault(r, []).append(pos[t])
    for t, (typ, r, i, j) in enumerate(q.tolist()):
        deps = []
        if r >= 1:
            deps.append(at[(r - 1, i, j)])
        if typ in (1, 2):
            deps.append(at[(r, r, r)])
            if r >= 1:
                deps.append(at[(r - 1, r, r)])      # the fused task that closed the pivot
        if typ == 3:
            deps += [at[(r, i, r)], at[(r, r, j)]]
        if typ == 0 and r >= 2:
            deps += p2.get(r - 2, [])
        if typ == 3 and i == j == r + 1 and r >= 1:
            deps += p2.get(r - 1, [])               # the fused pivot's snapshot slot
        if typ in (1, 2) and r >= 2:
            deps += p3.get(r - 2, [])
        for d in deps:
            assert d < pos[t], (q[t].tolist(), d, pos[t])


@pytest.mark.parametrize("seed", [0, 1, 7, 2 ** 63 + 5])
def test_batched_task_list_orders(fw, seed):
    """The batched plan's claim order (host only): every task of every graph
    exactly once, each graph's dependencies in order -- with the planned
    order (seed 0) and with the debug shuffle, which permutes each wave
    segment (a different order for every seed, the same tasks)."""
    ns = [700, 64, 300, 1000, 129, 33, 513]
    bss = [64, 32, 32, 128, 64, 32, 128]
    lst = fw.fw_batched_task_list(ns, bss, sms=152, options=fw.Options.default(debug_shuffle=seed))
    Rs = [-(-n // b) for n, b in zip(ns, bss)]
    assert len(lst) == sum(R ** 3 for R in Rs)
    for g, (n, R) in enumerate(zip(ns, Rs)):
        mine = np.flatnonzero(lst[:, 0] == g)
        ts = lst[mine, 1]
        assert sorted(ts.tolist()) == list(range(R ** 3))
        look = fw.fw_solve_plan(n, fw.Options.default(bs=bss[g]), sms=152)["lookahead"]
        q = fw.fw_queue_tasks(R, look)
        pos = np.empty(R ** 3, np.int64)
        pos[ts] = mine
        _check_order(q, pos)
    plain = fw.fw_batched_task_list(ns, bss, sms=152)
    # the checker fails a planted mistake: graph 3's first panel claimed
    # before its pivot
    R3 = Rs[3]
    q3 = fw.fw_queue_tasks(R3, fw.fw_solve_plan(ns[3], fw.Options.default(bs=bss[3]),
                                                sms=152)["lookahead"])
    mine = np.flatnonzero(plain[:, 0] == 3)
    pos = np.empty(R3 ** 3, np.int64)
    pos[plain[mine, 1]] = mine
    piv = int(np.flatnonzero((q3[:, 0] == 0) & (q3[:, 1] == 0))[0])
    pan = int(np.flatnonzero((q3[:, 0] == 1) & (q3[:, 1] == 0))[0])
    pos[piv], pos[pan] = pos[pan], pos[piv]
    with pytest.raises(AssertionError):
        _check_order(q3, pos)
    if seed:
        assert not np.array_equal(lst, plain)
        other = fw.fw_batched_task_list(ns, bss, sms=152,
                                        options=fw.Options.default(debug_shuffle=seed + 1))
        assert not np.array_equal(lst, other)
    else:
        assert np.array_equal(lst, plain)


def test_batched_task_list_checks(fw):
    lib = fw.load()
    import ctypes as C
    ns = np.array([100, 40], np.int64)
    bs = np.array([32, 64], np.int32)
    out = np.zeros((64 + 1, 2), np.int32)
    cnt = C.c_int64()
    assert lib.fw_batched_task_list(ns.ctypes.data, bs.ctypes.data, 2, 152, None,
                                    out.ctypes.data, 65, C.byref(cnt)) == 0 and cnt.value == 65
    assert lib.fw_batched_task_list(ns.ctypes.data, bs.ctypes.data, 2, 152, None,
                                    out.ctypes.data, 64, C.byref(cnt)) == 1    # cap too small
    bad = np.array([32, 48], np.int32)
    assert lib.fw_batched_task_list(ns.ctypes.data, bad.ctypes.data, 2, 152, None,
                                    out.ctypes.data, 65, C.byref(cnt)) == 1
    assert lib.fw_batched_task_list(ns.ctypes.data, bs.ctypes.data, 2, 0, None,
                                    out.ctypes.data, 65, C.byref(cnt)) == 1    # sms < 1
    assert lib.fw_batched_task_list(None, bs.ctypes.data, 2, 152, None,
                                    out.ctypes.data, 65, C.byref(cnt)) == 1


def test_batched_host_checks(fw):
    lib = fw.load()
    import ctypes as C
    h = C.c_void_p()
    ns = np.array([10, 20], np.int64)
    lds = np.array([12, 20], np.int64)
    assert lib.fw_batched_plan_create(C.byref(h), ns.ctypes.data, lds.ctypes.data, 0, 0, None) == 1
    bad = np.array([12, 18], np.int64)   # ld % 4 != 0
    assert lib.fw_batched_plan_create(C.byref(h), ns.ctypes.data, bad.ctypes.data, 2, 0, None) == 1
    small = np.array([8, 20], np.int64)  # ld < n
    assert lib.fw_batched_plan_create(C.byref(h), ns.ctypes.data, small.ctypes.data, 2, 0, None) == 1
    o = fw.Options.default(bs=96)
    assert lib.fw_batched_plan_create(C.byref(h), ns.ctypes.data, lds.ctypes.data, 2, 0,
                                      C.byref(o)) == 1
    assert lib.fw_solve_batched(None, None, None, None) == 1


def test_bs_table_host(fw):
    """One table per element type (the 64-bit types have no batched path);
    writing one leaves the other alone."""
    ti, tf = fw.fw_bs_table(), fw.fw_bs_table(dtype=fw.FW_F32)
    for t in (ti, tf):
        assert len(t) == 7 and set(t.tolist()) <= {32, 64, 128}
    with pytest.raises(fw.FWError):
        fw.fw_bs_table(np.array([32, 32, 48, 64, 128, 128, 128], np.int32))
    for dt in (fw.FW_I64, fw.FW_F64, 7):
        with pytest.raises(fw.FWError):
            fw.fw_bs_table(dtype=dt)
    other = np.array([32, 32, 32, 32, 32, 32, 32], np.int32)
    fw.fw_bs_table(other, dtype=fw.FW_F32)
    assert (fw.fw_bs_table(dtype=fw.FW_F32) == other).all()
    assert (fw.fw_bs_table() == ti).all()
    fw.fw_bs_table(tf, dtype=fw.FW_F32)
    fw.fw_bs_table(ti)
    assert (fw.fw_bs_table() == ti).all() and (fw.fw_bs_table(dtype=fw.FW_F32) == tf).all()


def test_solve_plan_choices(fw):
    """fw_solve_plan (host only): the automatic block size and lookahead, the
    rounds and the workspace a solve keeps, and its argument checks."""
    p = fw.fw_solve_plan(32768, sms=152)
    assert p["bs"] == 128 and p["rounds"] == 256 and p["lookahead"] == 6 * 152
    # snapshots dominate: 2 slots x R x BS^2 x 4 B x 5 arrays = 160 MiB (+ flags, offsets)
    assert 5 * 2 * 256 * 128 * 128 * 4 <= p["workspace_bytes"] < 170 * 2 ** 20
    assert fw.fw_solve_plan(512)["bs"] == 32
    assert fw.fw_solve_plan(3072)["bs"] == 64 and fw.fw_solve_plan(3073)["bs"] == 128
    # few tasks per round: at least 3 x SMs stay behind the panels, at least 2 x SMs ahead
    p = fw.fw_solve_plan(4096, fw.Options.default(bs=128), sms=152)
    assert p["rounds"] == 32 and p["lookahead"] == 31 * 31 - 61 - 3 * 152
    p = fw.fw_solve_plan(1024, fw.Options.default(bs=128), sms=152)
    assert p["lookahead"] == 2 * 152
    assert fw.fw_solve_plan(8192, fw.Options.default(lookahead=77))["lookahead"] == 77
    # 64-bit elements: BS 64 above 512 vertices, no BS = 128, snapshots of 8-byte
    # elements without the packed keys
    for dt in (fw.FW_I64, fw.FW_F64):
        p8 = fw.fw_solve_plan(8192, sms=152, dtype=dt)
        assert p8["bs"] == 64 and p8["rounds"] == 128
        assert fw.fw_solve_plan(300, dtype=dt)["bs"] == 32
        with pytest.raises(fw.FWError) as e:
            fw.fw_solve_plan(8192, fw.Options.default(bs=128), dtype=dt)
        assert e.value.code == 6
    p4 = fw.fw_solve_plan(8192, fw.Options.default(bs=64), sms=152)
    p8 = fw.fw_solve_plan(8192, fw.Options.default(bs=64), sms=152, dtype=fw.FW_F64)
    assert p8["workspace_bytes"] != p4["workspace_bytes"]
    lib = fw.load()
    assert lib.fw_solve_plan(0, fw.FW_I32, None, 152, None, None, None, None) == 1
    assert lib.fw_solve_plan(100, fw.FW_I32, None, 0, None, None, None, None) == 1
    assert lib.fw_solve_plan(100, 9, None, 152, None, None, None, None) == 1
    assert lib.fw_solve_plan(131072, fw.FW_I32, ctypes.byref(fw.Options.default(bs=32)), 152,
                             None, None, None, None) == 6


def test_paths_argument_checks(fw):
    """fw_paths rejects bad arguments on the host and launches nothing for an
    empty batch (no GPU needed)."""
    lib = fw.load()
    p = ctypes.c_void_p(16)
    assert lib.fw_paths(None, 10, 10, p, p, 1, p, 4, p, None) == 1
    assert lib.fw_paths(p, 0, 10, p, p, 1, p, 4, p, None) == 1
    assert lib.fw_paths(p, 10, 8, p, p, 1, p, 4, p, None) == 1
    assert lib.fw_paths(p, 10, 10, p, p, -1, p, 4, p, None) == 1
    assert lib.fw_paths(p, 10, 10, p, p, 1, p, 0, p, None) == 1
    assert lib.fw_paths(p, 10, 10, p, p, 0, p, 4, p, None) == 0


def test_host_io_argument_checks(fw):
    """fw_solve_host_io's host checks: null weights or distance buffers, and
    the in-place entry point's own checks (no CUDA call is reached)."""
    lib = fw.load()
    p = ctypes.c_void_p(16)
    assert lib.fw_solve_host_io(None, p, None, 10, 12, fw.FW_I32, None, None) == 1
    assert lib.fw_solve_host_io(p, None, None, 10, 12, fw.FW_I32, None, None) == 1
    assert lib.fw_solve_host_io(p, p, None, 0, 12, fw.FW_I32, None, None) == 1
    assert lib.fw_solve_host_io(p, p, None, 10, 10, fw.FW_I32, None, None) == 1   # ld % 4
    assert lib.fw_solve_host_io(p, p, None, 10, 12, 9, None, None) == 1
    assert lib.fw_solve_host(None, None, 10, 12, fw.FW_I32, None, None) == 1


def test_intermediate_argument_checks(fw):
    """fw_intermediate's host checks (no launch; batch 0 is a no-op)."""
    lib = fw.load()
    p = ctypes.c_void_p(16)
    assert lib.fw_intermediate(None, p, 10, 10, 1, 100, None) == 1
    assert lib.fw_intermediate(p, None, 10, 10, 1, 100, None) == 1
    assert lib.fw_intermediate(p, p, 0, 10, 1, 100, None) == 1
    assert lib.fw_intermediate(p, p, 10, 8, 1, 100, None) == 1
    assert lib.fw_intermediate(p, p, 10, 12, -1, 120, None) == 1
    assert lib.fw_intermediate(p, p, 10, 12, 2, 119, None) == 1     # stride < n * ld
    assert lib.fw_intermediate(p, p, 57345, 57348, 1, 0, None) == 6
    assert lib.fw_intermediate(p, p, 50000, 50000, 50000, 50000 * 50000, None) == 1
    assert lib.fw_intermediate(p, p, 10, 12, 0, 0, None) == 0


def test_wide_dtype_and_tile_call_host_checks(fw):
    """Checks made on the host before any CUDA call: 64-bit dtypes take BS 32
    or 64, and the tile-level calls reject bad block sizes, dtypes, leading
    dimensions, misalignment and the overlaps they do not allow."""
    lib = fw.load()
    g = 0x10000  # never dereferenced
    o = fw.Options.default(bs=128)
    for dt in (fw.FW_I64, fw.FW_F64):
        assert lib.fw_solve_ex(g, g + 4096, 8, 8, dt, ctypes.byref(o), None) == 6
    # fw_tile_closure
    assert lib.fw_tile_closure(g, g + 65536, 64, 48, fw.FW_I32, None) == 1     # bs
    assert lib.fw_tile_closure(g, g + 65536, 64, 64, 9, None) == 1             # dtype
    assert lib.fw_tile_closure(g, g + 65536, 32, 64, fw.FW_I32, None) == 1     # ld < bs
    assert lib.fw_tile_closure(g + 4, g + 65536, 64, 64, fw.FW_I32, None) == 1  # misaligned
    assert lib.fw_tile_closure(g, g, 64, 64, fw.FW_I32, None) == 1              # pred == dist
    assert lib.fw_tile_closure(g, g + 65536, 128, 128, fw.FW_F64, None) == 6   # 64-bit bs 128
    # fw_tile_minplus(C, Pc, ldc, A, lda, B, ldb, Pb, ldpb, tm, tn, bs, si, sj, dtype, s)
    M = lib.fw_tile_minplus
    A, B, C, Pc, Pb = g, g + (1 << 20), g + (2 << 20), g + (3 << 20), g + (4 << 20)
    I32 = fw.FW_I32
    assert M(C, Pc, 128, A, 32, B, 128, None, 128, 2, 4, 32, -1, -1, I32, None) == 1  # Pb missing
    assert M(C, Pc, 64, A, 32, B, 128, Pb, 128, 2, 4, 32, -1, -1, I32, None) == 1     # ldc < 4 bs
    assert M(C, Pc, 128, A, 32, B, 128, Pb, 128, 2, 4, 48, -1, -1, I32, None) == 1    # bs
    assert M(C, Pc, 130, A, 32, B, 128, Pb, 128, 2, 4, 32, -1, -1, I32, None) == 1    # ld % 4
    assert M(C + 8, Pc, 128, A, 32, B, 128, Pb, 128, 2, 4, 32, -1, -1, I32, None) == 1  # align
    # C may be A only with one tile column, B only with one tile row
    assert M(C, Pc, 128, C, 128, B, 128, Pb, 128, 2, 4, 32, -1, -1, I32, None) == 1
    assert M(C, Pc, 128, A, 32, C, 128, Pb, 128, 2, 4, 32, -1, -1, I32, None) == 1
    assert M(C, Pc, 128, A, 32, B, 128, Pc, 128, 2, 4, 32, -1, -1, I32, None) == 1
    assert M(C, Pc, 128, A, 32, B, 128, Pb, 128, 0, 4, 32, -1, -1, I32, None) == 0    # no tiles
    assert M(C, Pc, 128, A, 32, B, 128, Pb, 128, 2, 4, 128, -1, -1, fw.FW_F64, None) == 6
    assert lib.fw_block_init_pred(None, g, 8, 8, 8, 32, 8, 0, 1, 0, 1, I32, None) == 1
    assert lib.fw_block_init_pred(g, g + 4096, 8, 0, 8, 32, 8, 0, 1, 0, 1, I32, None) == 0
