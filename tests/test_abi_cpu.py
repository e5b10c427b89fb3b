"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every symbol include/ndg.h declares, sizes workspaces, and rejects bad
arguments before launching anything."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ndg():
    from paper_2405_20067_gb300 import build, ndg
    build.build()
    return ndg


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ndg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ndg_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(ndg):
    names = declared_functions()
    assert len(names) >= 10
    L = ndg.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(names) == sorted(ndg.EXPORTS)


def test_version_and_status_strings(ndg):
    assert ndg.lib().ndg_version() == 1
    assert ndg.status_string(0) == "ok"
    assert "capacity" in ndg.status_string(2)


def _mix_c(ndg, N=6, G=10, G_cap=10):
    fake = ctypes.c_void_p(0x1000)
    return ndg.MixtureC(N, G, G_cap, 0, fake, fake, fake, fake, None, None, None, None)


def test_workspace_size_grows_with_capacity(ndg):
    L = ndg.lib()
    m = _mix_c(ndg)
    q = ndg.QueriesC(1000, 256, ctypes.c_void_p(0x2000))
    cp = ndg.CullParamsC(16, ctypes.c_void_p(0x3000), 1.0 / 255, 3.0, 64)
    a = L.ndg_workspace_size(ctypes.byref(m), ctypes.byref(q), ctypes.byref(cp), 0)
    b = L.ndg_workspace_size(ctypes.byref(m), ctypes.byref(q), ctypes.byref(cp), 10_000)
    assert 0 < a < b
    bad = _mix_c(ndg, N=13)
    assert L.ndg_workspace_size(ctypes.byref(bad), None, None, 0) == 0


def test_invalid_arguments_rejected_on_host(ndg):
    """Each case fails argument validation before any CUDA call."""
    L = ndg.lib()
    ws = ctypes.c_void_p(0x100000)
    q = ndg.QueriesC(100, 256, ctypes.c_void_p(0x2000))
    cp = ndg.CullParamsC(4, ctypes.c_void_p(0x3000), 0.0, 3.0, 64)
    cull = ndg.CullC(ctypes.c_void_p(0x4000), ctypes.c_void_p(0x5000), 100, ctypes.c_void_p(0x6000))
    BIG = 1 << 40
    cases = [
        (_mix_c(ndg, N=0), q, cp),                       # N out of range
        (_mix_c(ndg, N=13), q, cp),                      # N out of range
        (_mix_c(ndg, G=11, G_cap=10), q, cp),            # G > G_cap
        (_mix_c(ndg), ndg.QueriesC(100, 0, ctypes.c_void_p(0x2000)), cp),    # tile 0
        (_mix_c(ndg), ndg.QueriesC(100, 257, ctypes.c_void_p(0x2000)), cp),  # tile > 256
        (_mix_c(ndg), ndg.QueriesC(100, 256, None), cp),                      # x NULL
        (_mix_c(ndg), q, ndg.CullParamsC(33, ctypes.c_void_p(0x3000), 0.0, 3.0, 64)),  # k > 32
        (_mix_c(ndg), q, ndg.CullParamsC(4, None, 0.0, 3.0, 64)),                      # proj NULL
        (_mix_c(ndg), q, ndg.CullParamsC(4, ctypes.c_void_p(0x3000), 0.0, 3.0, 256)),  # B > 255
        (_mix_c(ndg), q, ndg.CullParamsC(4, ctypes.c_void_p(0x3000), -1.0, 3.0, 64)),  # cutoff < 0
        (_mix_c(ndg), q, ndg.CullParamsC(4, ctypes.c_void_p(0x3000), 0.0, 3.0, 64, -1.0)),  # floor < 0
    ]
    for m, qq, cc in cases:
        st = L.ndg_build_cull(ctypes.byref(m), ctypes.byref(qq), ctypes.byref(cc),
                              ctypes.byref(cull), ws, BIG, None, None)
        assert st == 1, (m.N, m.G, qq.tile_size, cc.k)
    # misaligned workspace and a workspace that is too small
    m = _mix_c(ndg)
    assert L.ndg_build_cull(ctypes.byref(m), ctypes.byref(q), ctypes.byref(cp), ctypes.byref(cull),
                            ctypes.c_void_p(0x100010), BIG, None, None) == 1
    assert L.ndg_build_cull(ctypes.byref(m), ctypes.byref(q), ctypes.byref(cp), ctypes.byref(cull),
                            ws, 1024, None, None) == 6
    assert L.ndg_forward(ctypes.byref(m), ctypes.byref(q), ctypes.byref(cull), 7,
                         ctypes.c_void_p(0x7000), ws, BIG, None, None) == 1  # unknown mode
    assert L.ndg_loss_l2(-1, None, None, None, None, ws, BIG, None, None) == 1
    assert L.ndg_loss_rel_l2(10, ctypes.c_void_p(0x7000), ctypes.c_void_p(0x8000), 0.0,
                             ctypes.c_void_p(0x9000), ctypes.c_void_p(0xa000), ws, BIG, None,
                             None) == 1  # eps must be > 0
    assert L.ndg_selftest_timeout(2, ws, BIG, None) == 1  # unknown wait kind


def test_backward_order_host_checks(ndg):
    """ndg_backward_order applies ndg_backward's argument and workspace rules
    before any CUDA call; the order flag is the header's."""
    L = ndg.lib()
    src = open(os.path.join(ROOT, "include", "ndg.h")).read()
    flag = int(re.search(r"#define\s+NDG_BWD_ORDER_READY\s+(0x[0-9a-fA-F]+|\d+)", src).group(1), 0)
    assert flag == ndg.NDG_BWD_ORDER_READY
    assert flag & (ndg.NDG_MODE_FP32 | ndg.NDG_MODE_TC | ndg.NDG_MODE_AUTO) == 0
    rflag = int(re.search(r"#define\s+NDG_RECORDS_READY\s+(0x[0-9a-fA-F]+|\d+)", src).group(1), 0)
    assert rflag == ndg.NDG_RECORDS_READY
    assert rflag & (flag | ndg.NDG_MODE_FP32 | ndg.NDG_MODE_TC | ndg.NDG_MODE_AUTO) == 0
    m = _mix_c(ndg)
    q = ndg.QueriesC(100, 256, ctypes.c_void_p(0x2000))
    cull = ndg.CullC(ctypes.c_void_p(0x4000), ctypes.c_void_p(0x5000), 100, ctypes.c_void_p(0x6000))
    ws = ctypes.c_void_p(0x100000)
    BIG = 1 << 40
    E = ndg.NDG_ERR_INVALID_ARG
    assert L.ndg_backward_order(ctypes.byref(_mix_c(ndg, N=13)), ctypes.byref(q),
                                ctypes.byref(cull), ws, BIG, None, None) == E
    assert L.ndg_backward_order(ctypes.byref(m), ctypes.byref(q), ctypes.byref(cull), None, BIG,
                                None, None) == E
    assert L.ndg_backward_order(ctypes.byref(m), ctypes.byref(q), ctypes.byref(cull),
                                ctypes.c_void_p(0x100010), BIG, None, None) == E
    huge = ndg.CullC(ctypes.c_void_p(0x4000), ctypes.c_void_p(0x5000), 1 << 31,
                     ctypes.c_void_p(0x6000))
    assert L.ndg_backward_order(ctypes.byref(m), ctypes.byref(q), ctypes.byref(huge), ws, BIG,
                                None, None) == E  # E_cap must stay below 2^31
    assert L.ndg_backward_order(ctypes.byref(m), ctypes.byref(q), ctypes.byref(cull), ws, 1024,
                                None, None) == ndg.NDG_ERR_WORKSPACE


def test_mode_constants_match_header(ndg):
    """The binding's mode numbers and AUTO threshold are the header's."""
    import os
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "ndg.h")).read()
    defs = dict(re.findall(r"#define\s+(NDG_[A-Z_0-9]+)\s+(\d+)", src))
    assert int(defs["NDG_MODE_FP32"]) == ndg.NDG_MODE_FP32
    assert int(defs["NDG_MODE_TC"]) == ndg.NDG_MODE_TC
    assert int(defs["NDG_MODE_AUTO"]) == ndg.NDG_MODE_AUTO
    m = re.search(r"#define\s+NDG_AUTO_MIN_CANDIDATES\(N\)\s+\(\(N\) <= (\d+) \? (\d+) : (\d+)\)", src)
    lim, lo, hi = (int(v) for v in m.groups())
    for N in range(1, 13):
        assert ndg.auto_min_candidates(N) == (lo if N <= lim else hi), N


def test_noalloc_rejects_bad_pointers_on_host(ndg):
    """ndg_forward_noalloc applies ndg_forward's argument rules (NULL and
    misaligned FP32 pointers, sizes) before any CUDA call, so a bad pointer
    is an error status, never a launch."""
    L = ndg.lib()
    q = ndg.QueriesC(100, 256, ctypes.c_void_p(0x2000))
    cull = ndg.CullC(ctypes.c_void_p(0x4000), ctypes.c_void_p(0x5000), 100, None)
    y = ctypes.c_void_p(0x7000)
    fake = ctypes.c_void_p(0x1000)
    odd = ctypes.c_void_p(0x1002)  # not 4-byte aligned
    for i in range(4):  # each parent parameter misaligned in turn
        ptrs = [fake] * 4
        ptrs[i] = odd
        m = ndg.MixtureC(6, 10, 10, 0, *ptrs, None, None, None, None)
        assert L.ndg_forward_noalloc(ctypes.byref(m), ctypes.byref(q), ctypes.byref(cull), y,
                                     None) == 1, i
    for i in range(4):  # each child parameter misaligned in turn
        ch = [fake] * 4
        ch[i] = odd
        m = ndg.MixtureC(6, 10, 10, 1, fake, fake, fake, fake, *ch)
        assert L.ndg_forward_noalloc(ctypes.byref(m), ctypes.byref(q), ctypes.byref(cull), y,
                                     None) == 1, i
    m = _mix_c(ndg)
    bad_q = ndg.QueriesC(100, 256, ctypes.c_void_p(0x2001))
    assert L.ndg_forward_noalloc(ctypes.byref(m), ctypes.byref(bad_q), ctypes.byref(cull), y,
                                 None) == 1
    assert L.ndg_forward_noalloc(ctypes.byref(m), ctypes.byref(q), ctypes.byref(cull),
                                 ctypes.c_void_p(0x7002), None) == 1  # y misaligned
    bad_cull = ndg.CullC(ctypes.c_void_p(0x4004), ctypes.c_void_p(0x5000), 100, None)
    assert L.ndg_forward_noalloc(ctypes.byref(m), ctypes.byref(q), ctypes.byref(bad_cull), y,
                                 None) == 1  # int64 offsets misaligned
    bad_ids = ndg.CullC(ctypes.c_void_p(0x4000), ctypes.c_void_p(0x5002), 100, None)
    assert L.ndg_forward_noalloc(ctypes.byref(m), ctypes.byref(q), ctypes.byref(bad_ids), y,
                                 None) == 1
    assert L.ndg_forward_noalloc(ctypes.byref(_mix_c(ndg, N=13)), ctypes.byref(q),
                                 ctypes.byref(cull), y, None) == 1
    # beyond the fixed scratch: refused before any launch as well
    big = ndg.MixtureC(6, 200_000, 200_000, 0, fake, fake, fake, fake, None, None, None, None)
    assert L.ndg_forward_noalloc(ctypes.byref(big), ctypes.byref(q), ctypes.byref(cull), y,
                                 None) == ndg.NDG_ERR_SCRATCH_LIMIT


def test_forward_batch_host_checks(ndg):
    """ndg_forward_batch sizes its descriptor workspace and rejects bad
    arguments of any frame before any CUDA call."""
    L = ndg.lib()
    assert L.ndg_batch_workspace_size(0) == 0
    s1, s64 = L.ndg_batch_workspace_size(1), L.ndg_batch_workspace_size(64)
    assert 0 < s1 < s64 and s64 % 256 == 0
    m = _mix_c(ndg)
    q = ndg.QueriesC(1000, 256, ctypes.c_void_p(0x2000))
    c = ndg.CullC(ctypes.c_void_p(0x4000), ctypes.c_void_p(0x5000), 100, ctypes.c_void_p(0x6000))
    fake_ws = ctypes.c_void_p(0x10000)

    def frames(*fs):
        arr = (ndg.FrameC * len(fs))()
        for i, (mm, y, ws, nb) in enumerate(fs):
            arr[i] = ndg.FrameC(ctypes.pointer(mm), ctypes.pointer(q), ctypes.pointer(c), y, ws, nb)
        return arr

    good = (m, 0x7000, 0x10000, 1 << 30)
    bad_n = _mix_c(ndg, N=13)
    E = ndg.NDG_ERR_INVALID_ARG
    # no frames, no descriptor workspace, misaligned descriptor workspace
    assert L.ndg_forward_batch(frames(good), 0, fake_ws, s1, None, None, None) == E
    assert L.ndg_forward_batch(frames(good), 1, None, s1, None, None, None) == E
    assert L.ndg_forward_batch(frames(good), 1, ctypes.c_void_p(0x10010), s1, None, None, None) == E
    # descriptor workspace too small
    assert L.ndg_forward_batch(frames(good, good), 2, fake_ws, s1 - 256, None, None,
                               None) == ndg.NDG_ERR_WORKSPACE
    # a bad second frame: N out of range, no output, misaligned or short workspace
    for f2 in [(bad_n, 0x7000, 0x10000, 1 << 30), (m, None, 0x10000, 1 << 30),
               (m, 0x7000, 0x10008, 1 << 30)]:
        assert L.ndg_forward_batch(frames(good, f2), 2, fake_ws, s64, None, None, None) == E
    assert L.ndg_forward_batch(frames(good, (m, 0x7000, 0x10000, 16)), 2, fake_ws, s64, None,
                               None, None) == ndg.NDG_ERR_WORKSPACE
    # an unknown frame flag
    fs = frames(good, good)
    fs[1].flags = 0x4
    assert L.ndg_forward_batch(fs, 2, fake_ws, s64, None, None, None) == E
