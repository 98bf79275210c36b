"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every function
that include/peps_vmc.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2409_05285_gb300 import binding
from paper_2409_05285_gb300.build import LIB, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(peps_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    build()
    assert os.path.exists(LIB)
    lib = ctypes.CDLL(LIB)
    names = declared_functions()
    assert "peps_init" in names and "peps_sr_step" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(binding.EXPORTS) <= set(names)


def test_binding_loads_and_reports_version():
    lib = binding.load()
    assert lib.peps_version().startswith(b"peps_vmc")
    assert lib.peps_last_error(None) == b""


def test_invalid_params_rejected_without_gpu_work():
    lib = binding.load()
    p = binding.Params(L1=1, L2=4, model=0, J1=1.0, J2=0.0, D=2, chi=4, n_chains=4,
                       precision=0, init_noise=1e-3, seed=0, n_blocks=0)
    ctx = ctypes.c_void_p()
    assert lib.peps_init(ctypes.byref(p), None, ctypes.byref(ctx)) == binding.PEPS_EINVAL
    p.L1, p.chi = 4, 65
    assert lib.peps_init(ctypes.byref(p), None, ctypes.byref(ctx)) == binding.PEPS_EINVAL
    p.chi, p.precision = 4, 7
    assert lib.peps_init(ctypes.byref(p), None, ctypes.byref(ctx)) == binding.PEPS_EINVAL
    assert not ctx.value


def test_footprint_is_host_arithmetic():
    # admission by footprint needs no device work: 0 for invalid parameters, and the bytes
    # grow with the chain count (chain-outermost buffers) and with chi
    lib = binding.load()
    lib.peps_footprint.restype = ctypes.c_size_t
    p = binding.Params(L1=8, L2=8, model=0, J1=1.0, J2=0.0, D=4, chi=16, n_chains=8192,
                       precision=binding.PEPS_TF32, init_noise=1e-3, seed=0, n_blocks=0)
    big = lib.peps_footprint(ctypes.byref(p))
    p.n_chains = 4096
    half = lib.peps_footprint(ctypes.byref(p))
    assert 0 < half < big <= 2 * half + (1 << 26)
    p.chi = 8
    assert lib.peps_footprint(ctypes.byref(p)) < half
    p.L1 = 1
    assert lib.peps_footprint(ctypes.byref(p)) == 0


def test_tuning_and_profile_calls_reject_a_null_context():
    lib = binding.load()
    t = binding.Tune(grid_pct=100, db_bytes=0, ffma_g=16, kc_max=64)
    assert lib.peps_set_tune(None, ctypes.byref(t)) == binding.PEPS_EINVAL
    assert lib.peps_autotune(None, 0, ctypes.byref(t)) == binding.PEPS_EINVAL
    buf = (ctypes.c_double * 4)()
    n = ctypes.c_int()
    assert lib.peps_profile_launch_bytes(None, b"kb_gemm_tc", buf, 4, ctypes.byref(n)) == \
        binding.PEPS_EINVAL


def test_direct_calls_reject_a_null_context_and_next_bd_follows_the_oracle():
    # host-only arithmetic of the direct sampler's diagonal bias against the oracle's rule
    import numpy as np
    from oracle import direct
    lib = binding.load()
    bd = ctypes.c_double(0.5)
    assert lib.peps_direct_draw(None, None, 0, 0.5, 0.5, None) == binding.PEPS_EINVAL
    assert lib.peps_direct_step(None, ctypes.byref(bd), 0.5, 0.01, 1e-4, 10, 1e-8, None) == \
        binding.PEPS_EINVAL
    N = 6
    for b_d in (1.0, 0.7, 0.05):
        for n_diag in range(0, 11):
            S = np.vstack([np.zeros((n_diag, N), np.int64), np.ones((10 - n_diag, N), np.int64)])
            f = direct.diagonal_fraction(S)
            assert binding.direct_next_bd(b_d, f, N) == pytest.approx(
                direct.update_bd(b_d, S, N), rel=1e-15)


def test_group_calls_reject_bad_arguments_without_gpu_work():
    lib = binding.load()
    out = ctypes.c_void_p()
    assert lib.peps_group_create(None, 0, ctypes.byref(out)) == binding.PEPS_EINVAL
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.peps_group_create(arr, 1, ctypes.byref(out)) == binding.PEPS_EINVAL
    assert not out.value
    assert lib.peps_group_eval(None) == binding.PEPS_EINVAL
    lib.peps_group_free(None)


def test_header_is_plain_c():
    # the boundary is a C ABI: the header compiles as C99 (no C++ or torch types)
    import shutil
    import subprocess
    import pytest
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            subprocess.run([cc, "-fsyntax-only", "-x", "c", "-std=c99", "-Wall", "-Werror",
                            os.path.join(ROOT, "include", fn)], check=True)


def test_fermion_calls_reject_a_null_evaluator_and_init_theta_is_the_identity():
    # host-only: the fermionic calls refuse a null evaluator; the beta = 0 parameters equal
    # the oracle's |I> (noise 0), and with noise the parity-even entries carry the oracle's
    # own Philox draws, the parity-odd ones stay zero
    import numpy as np
    from oracle import fermion as fm
    from oracle import philox
    lib = binding.load()
    assert lib.peps_famp_n_moves(None) == binding.PEPS_EINVAL
    assert lib.peps_famp_sweep(None, None, 0, None, 0, 2, 1, 0, 0, None, None, None, None) == \
        binding.PEPS_EINVAL
    assert lib.peps_famp_sr_step(None, None, 0, None, 1, 1.0, 8.0, 4.0, 2, 0.01, 1e-4, 10,
                                 1e-8, None) == binding.PEPS_EINVAL
    assert lib.peps_famp_profile(None, 1) == binding.PEPS_EINVAL
    assert lib.peps_famp_set_strips(None, 1) == binding.PEPS_EINVAL
    assert lib.peps_famp_launches(None) == 0
    L1, L2, D = 2, 3, 2
    th = binding.famp_init_theta(L1, L2, D, noise=0.0, seed=3)
    off = 0
    for r in range(L1):
        for c in range(L2):
            dims = (1 if c == 0 else D, 1 if c == L2 - 1 else D, 1 if r == 0 else D, 1 if r == L1 - 1 else D)
            A = th[off:off + 16 * int(np.prod(dims))].reshape((16,) + dims)
            ref = np.zeros_like(A)
            ref[(slice(None), 0, 0, 0, 0)] = fm.identity_fpeps(1, 1)[0][:, 0, 0, 0, 0]
            assert np.array_equal(A, ref)
            off += A.size
    assert off == th.size
    a = 1e-3
    thn = binding.famp_init_theta(L1, L2, D, noise=a, seed=3)
    off = 0
    for i in range(L1 * L2):
        r, c = divmod(i, L2)
        dims = (1 if c == 0 else D, 1 if c == L2 - 1 else D, 1 if r == 0 else D, 1 if r == L1 - 1 else D)
        A = thn[off:off + 16 * int(np.prod(dims))].reshape((16,) + dims)
        for e, idx in enumerate(np.ndindex(*A.shape)):
            par = (bin(idx[0]).count("1") + sum(idx[1:])) & 1
            if par:
                assert A[idx] == 0.0
            elif all(x == 0 for x in idx[1:]) and (idx[0] & 3) == (idx[0] >> 2):
                assert A[idx] == th[off + e]
            else:
                u = philox.uniform(3, i, e, 0, 0x46494E54)
                assert A[idx] == pytest.approx(a * (2 * u - 1), rel=1e-15, abs=1e-300)
        off += A.size
    with pytest.raises(binding.PepsError):
        binding.famp_init_theta(L1, L2, D, noise=-1.0)


def test_fermion_move_table_is_the_oracle_sweep_order():
    # host-only: the device sweep's proposals, in order, are the oracle's (row phases: a row's
    # pairs and horizontal hops column by column, then its vertical hops)
    from oracle import fermion_vmc as fv
    for L1, L2 in ((2, 2), (2, 3), (3, 2), (4, 5), (6, 6)):
        t = binding.famp_move_table(L1, L2)
        ref = [(0, m[1], m[1], m[2]) if m[0] == "pair" else (1, m[1], m[2], m[3])
               for m in fv.moves(L1, L2)]
        assert [tuple(int(x) for x in row) for row in t] == ref, (L1, L2)
    assert binding.load().peps_famp_move_table(0, 2, None, 0) == binding.PEPS_EINVAL
