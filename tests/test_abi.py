"""The C-ABI library loads and exports every symbol that include/qrctm.h
declares; host-side planning and argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for f in os.listdir(INCLUDE):
        if f.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(INCLUDE, f)).read(), flags=re.S)
            names |= set(re.findall(r"\b(qrctm_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def q():
    from paper_2505_00494_b300 import build
    build.build()
    import paper_2505_00494_b300 as q
    return q


def test_every_declared_symbol_is_exported(q):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(q.lib, n), n
    assert set(names) == set(q.EXPORTED)   # the binding covers the whole header


def test_version(q):
    assert b"sm_103a" in q.lib.qrctm_version()


def cfg(q, d=2, D=6, chi=144, **kw):
    c = q.Config(d, D, chi, 0, 0, 0, 1, 1e-10, 500, 0, 0.0, 0, 0, None)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def test_workspace_planning_host_only(q):
    c = cfg(q)
    b1 = q.lib.qrctm_workspace_bytes(ctypes.byref(c))
    assert b1 > 0 and b1 % 256 == 0
    # at least X1, Z, X2 and the open-leg energy buffer (chi D^2)^2 (1 + d + 1 + d^2)
    m = 144 * 36
    assert b1 >= 8 * m * m * 8
    c.with_nnn = 1
    assert q.lib.qrctm_workspace_bytes(ctypes.byref(c)) > b1
    for bad in (cfg(q, chi=0), cfg(q, chi=2000), cfg(q, chi=16), cfg(q, precision=7),
                cfg(q, warmup_steps=-2)):
        assert q.lib.qrctm_workspace_bytes(ctypes.byref(bad)) == 0
    assert q.lib.qrctm_qr_workspace_bytes(10, 20) == 0
    assert q.lib.qrctm_qr_workspace_bytes(5184, 144) > 2 * 5184 * 144 * 8


def test_create_rejects_bad_arguments_without_gpu(q):
    c = cfg(q, D=2, chi=16)
    h = ctypes.c_void_p()
    assert q.lib.qrctm_create(ctypes.byref(c), None, 0, ctypes.byref(h)) == 1
    buf = ctypes.create_string_buffer(2048)
    aligned = (ctypes.addressof(buf) + 255) // 256 * 256
    assert q.lib.qrctm_create(ctypes.byref(c), ctypes.c_void_p(aligned + 8), 64,
                              ctypes.byref(h)) == 1
    assert q.lib.qrctm_create(ctypes.byref(c), ctypes.c_void_p(aligned), 256,
                              ctypes.byref(h)) == 6
    # null context calls fail cleanly
    assert q.lib.qrctm_step(None, 1, None) == 1
    assert q.lib.qrctm_householder_qr(4, 8, None, None, None, None, 0, None) == 1


def test_network_planning_host_only(q):
    # classical network mode: T's inner leg has D values, d = 1, FP64 only,
    # no energy/gradient buffers
    c = cfg(q, d=1, D=3, chi=27, layers=3)
    b = q.lib.qrctm_workspace_bytes(ctypes.byref(c))
    m = 27 * 3
    assert b > 0 and b >= 2 * m * m * 8
    assert b < q.lib.qrctm_workspace_bytes(ctypes.byref(cfg(q, d=1, D=3, chi=81, layers=3)))
    for bad in (cfg(q, d=2, D=3, chi=27, layers=3), cfg(q, d=1, D=3, chi=27, layers=3, precision=1),
                cfg(q, d=1, D=3, chi=27, layers=3, with_grad=1),
                cfg(q, d=1, D=3, chi=27, layers=3, with_nnn=1),
                cfg(q, d=1, D=3, chi=2, layers=3), cfg(q, d=1, D=3, chi=27, layers=4)):
        assert q.lib.qrctm_workspace_bytes(ctypes.byref(bad)) == 0
    assert q.lib.qrctm_init_env_network(None, None, None, None, None) == 1
    assert q.lib.qrctm_network_observables(None, None, None, None) == 1


def test_optimizer_planning_host_only(q):
    base = q.lib.qrctm_workspace_bytes(ctypes.byref(cfg(q, D=2, chi=16, with_grad=1)))
    with_opt = q.lib.qrctm_workspace_bytes(ctypes.byref(cfg(q, D=2, chi=16, with_grad=1,
                                                           opt_history=10)))
    # 2 x history x n pair vectors + 6 vectors + two environments
    n = 2 * 16
    assert with_opt >= base + (2 * 10 * n + 6 * n + 2 * (16 * 16 + 16 * 4 * 16)) * 8
    for bad in (cfg(q, D=2, chi=16, opt_history=10), cfg(q, D=2, chi=16, with_grad=1, opt_history=33),
                cfg(q, D=2, chi=16, with_grad=1, opt_history=-1)):
        assert q.lib.qrctm_workspace_bytes(ctypes.byref(bad)) == 0
    assert q.lib.qrctm_optimize(None, None, None, 1, None, None, None, None) == 1


def test_tape_store_planning_host_only(q):
    # the tapes of grad_store steps: each holds X1, Z, X2 (4 (chi D^2)^2 doubles at
    # d = 2) and a dozen environment-sized pieces; the reservation grows linearly
    ws = lambda n: q.lib.qrctm_workspace_bytes(ctypes.byref(cfg(q, D=3, chi=12, with_grad=1,
                                                                grad_store=n)))
    m = 12 * 9
    assert ws(1) - ws(0) >= 4 * m * m * 8
    assert ws(3) - ws(0) == 3 * (ws(1) - ws(0))   # every piece 256-byte aligned
    for bad in (cfg(q, D=3, chi=12, grad_store=2), cfg(q, D=3, chi=12, with_grad=1, grad_store=33),
                cfg(q, D=3, chi=12, with_grad=1, grad_store=-1)):
        assert q.lib.qrctm_workspace_bytes(ctypes.byref(bad)) == 0


def test_qr_width_limit_host_only(q):
    # one accumulator row per column of the factorisation: n <= 2048
    assert q.lib.qrctm_qr_workspace_bytes(4096, 2048) > 0
    assert q.lib.qrctm_qr_workspace_bytes(4096, 2049) == 0
