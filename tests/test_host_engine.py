"""The batched engine's orchestration (BatchRunner: environments, compression, strips,
ratios, O rows, Metropolis moves) built for the host over plain loops
(tests/host_engine/host_engine.cpp) and checked against the FP64 oracle on the CPU, with the
tolerances of the FP64 GPU parity tests.  The GPU kernels themselves are covered by the
`-m gpu` parity tests; this covers the sequence of operations without a GPU."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from oracle import peps, sampler
from oracle.lattice import Lattice
from paper_2409_05285_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host_engine", "host_engine.cpp")
CSRC = os.path.join(ROOT, "paper_2409_05285_gb300", "csrc")


@pytest.fixture(scope="module")
def engine(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("host_engine") / "host_engine")
    subprocess.run(["g++", "-std=c++17", "-O2", "-I", CSRC, SRC, "-o", exe], check=True)
    return exe


def _run(exe, tmp, mode, lat, chi, th, S, p=2, seed=0, sweep=0):
    n = S.shape[0]
    fin, fout = str(tmp / "in.bin"), str(tmp / "out.bin")
    with open(fin, "wb") as f:
        f.write(struct.pack("<7i", mode, lat.nrow, lat.ncol, lat.D, chi, n, p))
        f.write(struct.pack("<2d", lat.J1, lat.J2))
        f.write(struct.pack("<Qi", seed, sweep))
        f.write(np.asarray(th, dtype=np.float64).tobytes())
        f.write(np.asarray(S, dtype=np.uint8).tobytes())
    subprocess.run([exe, fin, fout], check=True)
    raw = open(fout, "rb").read()
    if mode in (6, 7):
        la = np.frombuffer(raw, np.float64, n, 0)
        sg = np.frombuffer(raw, np.int8, n, 8 * n)
        es = np.frombuffer(raw, np.float64, n, 9 * n)
        ea = np.frombuffer(raw, np.float64, n, 17 * n)
        if mode == 7:
            O = np.frombuffer(raw, np.float64, n * lat.No, 25 * n).reshape(n, lat.No)
            return la, sg, es, ea, O
        return la, sg, es, ea
    if mode == 5:
        S2 = np.frombuffer(raw, np.uint8, n * lat.N, 0).reshape(n, lat.N)
        acc = np.frombuffer(raw, np.int32, n, n * lat.N)
        return S2, acc
    if mode == 4:
        la = np.frombuffer(raw, np.float64, n, 0)
        sg = np.frombuffer(raw, np.int8, n, 8 * n)
        O = np.frombuffer(raw, np.float64, n * lat.No, 9 * n).reshape(n, lat.No)
        return la, sg, O
    if mode in (0, 3):
        o = 0
        la = np.frombuffer(raw, np.float64, n, o); o += 8 * n
        sg = np.frombuffer(raw, np.int8, n, o); o += n
        es = np.frombuffer(raw, np.float64, n, o); o += 8 * n
        ea = np.frombuffer(raw, np.float64, n, o); o += 8 * n
        O = np.frombuffer(raw, np.float64, n * lat.No, o).reshape(n, lat.No)
        return la, sg, es, ea, O
    N = lat.N
    S2 = np.frombuffer(raw, np.uint8, n * N, 0).reshape(n, N)
    acc = np.frombuffer(raw, np.int32, n, n * N)
    prop = np.frombuffer(raw, np.int32, n, n * N + 4 * n)
    return S2, acc, prop


CASES = [  # (L1, L2, D, chi, J2, n): exact chi (first two), truncated chi, NNN bonds
    (2, 2, 2, 4, 0.0, 4),
    (3, 3, 2, 4, 0.0, 5),
    (3, 4, 2, 3, 0.5, 4),
    (4, 3, 3, 5, 0.2, 3),
    (5, 4, 3, 6, 0.3, 2),
    (4, 6, 2, 3, 0.0, 2),
]


@pytest.mark.parametrize("case", CASES)
def test_host_engine_eval_matches_oracle(engine, tmp_path, case):
    L1, L2, D, chi, J2, n = case
    lat = Lattice(L1, L2, D, J1=1.0, J2=J2)
    th = wl.random_theta(L1, L2, D, seed=L1 * 10 + L2, scale=0.3, diag_bias=1.0)
    S = wl.random_configs(L1, L2, n, seed=D)
    la, sg, es, ea, O = _run(engine, tmp_path, 0, lat, chi, th, S)
    for k in range(n):
        r = peps.eval_sample(lat, th, S[k], chi)
        assert sg[k] == r['sign']
        assert abs(la[k] - r['log_abs']) <= 1e-10
        scale = max(1.0, abs(r['e_sys']), abs(r['e_anc']))
        assert abs(es[k] - r['e_sys']) <= 1e-9 * scale
        assert abs(ea[k] - r['e_anc']) <= 1e-9 * scale
        assert np.max(np.abs(O[k] - r['O'])) <= 1e-9 * max(1.0, np.max(np.abs(r['O'])))


@pytest.mark.parametrize("shape", [(3, 3, 2, 4, 0.0), (3, 4, 2, 3, 0.5), (4, 3, 3, 5, 0.2)])
@pytest.mark.parametrize("p", [2, 1])
def test_host_engine_sweep_matches_oracle(engine, tmp_path, p, shape):
    # one Metropolis sweep per chain with the same Philox stream: the same accepted moves
    # (exact chi, and a truncating chi with next-nearest-neighbour bonds)
    L1, L2, D, chi, J2 = shape
    lat = Lattice(L1, L2, D, J1=1.0, J2=J2)
    th = wl.random_theta(L1, L2, D, seed=33, scale=0.3, diag_bias=1.0)
    S = wl.random_configs(L1, L2, 6, seed=34)
    seed, sweep = 11, 5
    S2, acc, prop = _run(engine, tmp_path, 1, lat, chi, th, S, p=p, seed=seed, sweep=sweep)
    for ch in range(S.shape[0]):
        So, a, b = sampler.mc_sweep(lat, th, S[ch], chi, p, seed, ch, sweep)
        assert np.array_equal(S2[ch], So), ch
        assert (acc[ch], prop[ch]) == (a, b)


def test_host_engine_eval_heis8_shape(engine, tmp_path):
    # 8x8, D=4, chi=16: the bench workload's contraction sizes and truncations
    L, D, chi = 8, 4, 16
    lat = Lattice(L, L, D)
    th = wl.random_theta(L, L, D, seed=81, scale=0.2, diag_bias=1.0)
    S = wl.random_configs(L, L, 2, seed=82)
    la, sg, es, ea, O = _run(engine, tmp_path, 0, lat, chi, th, S)
    for k in range(S.shape[0]):
        r = peps.eval_sample(lat, th, S[k], chi)
        assert sg[k] == r['sign']
        assert abs(la[k] - r['log_abs']) <= 1e-10
        scale = max(1.0, abs(r['e_sys']), abs(r['e_anc']))
        assert abs(es[k] - r['e_sys']) <= 1e-9 * scale
        assert abs(ea[k] - r['e_anc']) <= 1e-9 * scale
        assert np.max(np.abs(O[k] - r['O'])) <= 1e-8 * max(1.0, np.max(np.abs(r['O'])))


def _run_draw(exe, tmp, lat, chi, th, u, b_d, expo):
    n, N = u.shape
    fin, fout = str(tmp / "in.bin"), str(tmp / "out.bin")
    with open(fin, "wb") as f:
        f.write(struct.pack("<7i", 2, lat.nrow, lat.ncol, lat.D, chi, n, 2))
        f.write(struct.pack("<2d", lat.J1, lat.J2))
        f.write(struct.pack("<Qi", 0, 0))
        f.write(np.asarray(th, dtype=np.float64).tobytes())
        f.write(np.zeros(n * N, dtype=np.uint8).tobytes())
        f.write(struct.pack("<2d", b_d, expo))
        f.write(np.asarray(u, dtype=np.float64).tobytes())
    subprocess.run([exe, fin, fout], check=True)
    raw = open(fout, "rb").read()
    return (np.frombuffer(raw, np.uint8, n * N, 0).reshape(n, N),
            np.frombuffer(raw, np.float64, n, n * N))


@pytest.mark.parametrize("case", [(2, 3, 2, 16, 1.0, 1.0), (3, 3, 2, 16, 0.4, 0.5),
                                  (3, 3, 2, 4, 0.6, 0.5), (3, 4, 2, 6, 1.0, 0.5)])
def test_host_engine_direct_draw_matches_oracle(engine, tmp_path, case):
    # reweighted direct sampling (App. A) through the engine's own environments and strips
    # over double-layer tensors (pv_direct.cuh) against the oracle's boundary-MPS form: the
    # same samples and log q for the same uniforms, at exact and at truncating chi
    from oracle import direct
    L1, L2, D, chi, b_d, expo = case
    lat = Lattice(L1, L2, D)
    th = wl.random_theta(L1, L2, D, seed=L1 * 7 + L2, scale=0.4, diag_bias=1.0)
    u = np.random.default_rng(L1 + 10 * L2 + chi).random((5, lat.N))
    S, lq = _run_draw(engine, tmp_path, lat, chi, th, u, b_d, expo)
    down = direct.summed_down_envs(lat, th, chi)
    for k in range(u.shape[0]):
        So, lqo = direct.draw_bmps(lat, th, u[k], chi, b_d, expo, down=down)
        assert np.array_equal(S[k], So), k
        assert lq[k] == pytest.approx(lqo, rel=1e-9, abs=1e-11)


@pytest.mark.parametrize("case", [(3, 4, 2, 3, 0.5, 4), (4, 3, 3, 5, 0.2, 3), (8, 8, 4, 16, 0.0, 2)])
def test_host_engine_gram_path_matches_oracle(engine, tmp_path, case):
    # the compression's right factors from the Gram matrices W W^T (the path the TF32 mode
    # takes on the GPU, here in float64 with a plain Cholesky): the truncation depends on the
    # factor only through L L^T, so the results match the oracle's Householder factors
    L1, L2, D, chi, J2, n = case
    lat = Lattice(L1, L2, D, J1=1.0, J2=J2)
    th = wl.random_theta(L1, L2, D, seed=L1 * 10 + L2, scale=0.3, diag_bias=1.0)
    S = wl.random_configs(L1, L2, n, seed=D)
    la, sg, es, ea, O = _run(engine, tmp_path, 3, lat, chi, th, S)
    for k in range(n):
        r = peps.eval_sample(lat, th, S[k], chi)
        assert sg[k] == r['sign']
        assert abs(la[k] - r['log_abs']) <= 1e-9
        scale = max(1.0, abs(r['e_sys']), abs(r['e_anc']))
        assert abs(es[k] - r['e_sys']) <= 1e-8 * scale
        assert abs(ea[k] - r['e_anc']) <= 1e-8 * scale
        assert np.max(np.abs(O[k] - r['O'])) <= 1e-7 * max(1.0, np.max(np.abs(r['O'])))


@pytest.mark.parametrize("case", [(2, 2, 3, 9, 4), (2, 3, 3, 9, 3), (3, 3, 2, 8, 3)])
def test_host_engine_fermion_plain_contraction_matches_oracle(engine, tmp_path, case):
    # the fermionic engine's form (pv_fermion.cuh, Fig. 1b): the plain boundary-MPS
    # contraction of the 32 signed slices per site at the extended indices S_i + 16 b_i, times
    # the configuration sign, is the fermionic amplitude; its plain O rows times each entry's
    # slice sign are the fermionic O.  Against the oracle's sums over every virtual assignment
    # at exact chi.
    from oracle import fermion as fm
    L1, L2, D, chi, n = case
    N = L1 * L2
    rng = np.random.default_rng(100 * L1 + 10 * L2 + D)
    T = fm.random_even_fpeps(L1, L2, D, rng, scale=0.7)
    th32 = np.concatenate([A.ravel() for A in fm.fpeps_signed_slices(T)])
    signs = fm.fpeps_signed_slices([np.ones_like(A) for A in T])
    S = rng.integers(0, 16, (n, N))
    for k in range(n):
        if sum(bin(int(x)).count("1") for x in S[k]) % 2:
            S[k, 0] ^= 1
    S32 = np.array([[int(S[k, i]) + 16 * b for i, b in enumerate(fm.fpeps_row_prefix_bits(L1, L2, S[k]))]
                    for k in range(n)], dtype=np.uint8)
    lat = Lattice(L1, L2, D)
    la, sg, O = _run(engine, tmp_path, 4, lat, chi, th32, S32)
    for k in range(n):
        grads, psi = fm.fpeps_log_derivative(L1, L2, T, S[k])
        assert psi == pytest.approx(fm.fpeps_amplitude_brute(L1, L2, T, S[k]), rel=1e-12)
        assert sg[k] * fm.fpeps_config_sign(L1, L2, S[k]) == np.sign(psi), k
        assert abs(la[k] - np.log(abs(psi))) <= 1e-10, k
        o = 0
        scale = max(1.0, max(np.max(np.abs(g)) for g in grads))
        for i in range(N):
            sz = grads[i].size
            plain = O[k, o:o + sz] * signs[i][S32[k, i]].ravel()
            assert np.max(np.abs(plain - grads[i].ravel())) <= 1e-9 * scale, (k, i)
            o += sz


@pytest.mark.parametrize("case,p", [((2, 2, 2, 4, 6), 2), ((3, 3, 2, 8, 6), 2), ((2, 3, 3, 9, 5), 1),
                                    ((3, 4, 2, 8, 4), 2)])
def test_host_engine_fermion_sweep_on_strips_matches_oracle(engine, tmp_path, case, p):
    # the fermionic sweep on cached one- and two-row strips (fermion_mc over 64 slices per
    # site: the signed slices and the same with a right-leg parity) against the oracle's sweep,
    # whose every proposal is a full contraction: the same Philox uniforms, the same decisions
    # (exact chi), so the same configurations and acceptance counts
    import functools
    from oracle import fermion as fm
    from oracle import fermion_vmc as fv
    L1, L2, D, chi, n = case
    N = L1 * L2
    rng = np.random.default_rng(7 * L1 + 3 * L2 + D + p)
    T = fm.random_even_fpeps(L1, L2, D, rng, scale=0.4)
    for i, A in enumerate(fm.identity_fpeps(L1, L2)):
        T[i][(slice(None), 0, 0, 0, 0)] += A[:, 0, 0, 0, 0]
    blocks = []
    for A in fm.fpeps_signed_slices(T):
        B = A.copy()
        B[:, :, 1::2, :, :] *= -1.0               # parity of the right leg
        blocks += [A.ravel(), B.ravel()]
    th64 = np.concatenate(blocks)
    a = rng.integers(0, 4, (n, N))
    S0 = (a | (a << 2)).astype(np.uint8)
    lat = Lattice(L1, L2, D)
    seed, sweep = 77, 3
    S, acc = _run(engine, tmp_path, 5, lat, chi, th64, S0, p=p, seed=seed, sweep=sweep)
    amp = functools.lru_cache(maxsize=None)(fm.fpeps_amplitude_function(L1, L2, T))
    M = len(fv.moves(L1, L2))
    margin = np.inf
    for c in range(n):
        x, a_ref, mg = fv.sweep(L1, L2, T, S0[c], p, fv.uniforms(seed, c, sweep, M),
                                amplitude=lambda X: amp(tuple(int(v) for v in X)))
        margin = min(margin, mg)
        assert np.array_equal(S[c], x), c
        assert acc[c] == a_ref, c
    assert margin > 1e-8
    assert acc.sum() > 0


def _fermion_th64(T):
    # the signed slices of every site followed by the same with a parity on the right leg
    from oracle import fermion as fm
    blocks = []
    for A in fm.fpeps_signed_slices(T):
        B = A.copy()
        B[:, :, 1::2, :, :] *= -1.0
        blocks += [A.ravel(), B.ravel()]
    return np.concatenate(blocks)


@pytest.mark.parametrize("case", [(2, 2, 2, 4, 6), (3, 3, 2, 8, 5), (2, 3, 3, 9, 4), (3, 4, 2, 8, 3)])
def test_host_engine_fermion_local_energy_on_strips_matches_oracle(engine, tmp_path, case):
    # fermion_eloc: every hop's ratio from a one-row (horizontal) or two-row (vertical) strip,
    # with the configuration-sign ratio, the Jordan-Wigner sign and a vertical hop's right-leg
    # sign, against the oracle's local energies (each hop a full row contraction), exact chi;
    # also log|psi| and the sign
    from oracle import fermion as fm
    L1, L2, D, chi, n = case
    N = L1 * L2
    t_hop, U, mu = 1.0, 8.0, 4.0
    rng = np.random.default_rng(11 * L1 + 5 * L2 + D)
    T = fm.random_even_fpeps(L1, L2, D, rng, scale=0.5)
    for i, A in enumerate(fm.identity_fpeps(L1, L2)):
        T[i][(slice(None), 0, 0, 0, 0)] += A[:, 0, 0, 0, 0]
    S = rng.integers(0, 16, (n, N))
    for k in range(n):
        if sum(bin(int(x)).count("1") for x in S[k]) % 2:
            S[k, 0] ^= 1
    S = S.astype(np.uint8)
    lat = Lattice(L1, L2, D, J1=t_hop, J2=U)
    mu_bits = struct.unpack("<Q", struct.pack("<d", mu))[0]
    la, sg, es, ea = _run(engine, tmp_path, 6, lat, chi, _fermion_th64(T), S, seed=mu_bits)
    for k in range(n):
        psi = fm.fpeps_amplitude_bosonic(L1, L2, T, S[k])
        assert sg[k] == np.sign(psi) and abs(la[k] - np.log(abs(psi))) <= 1e-10, k
        r_es, r_ea = fm.fpeps_local_energy(L1, L2, T, S[k], t_hop, U, mu)
        scale = max(1.0, abs(r_es), abs(r_ea))
        assert abs(es[k] - r_es) <= 1e-9 * scale, (k, es[k], r_es)
        assert abs(ea[k] - r_ea) <= 1e-9 * scale, (k, ea[k], r_ea)


@pytest.mark.parametrize("case", [(2, 2, 2, 4, 4), (3, 3, 2, 8, 3), (2, 3, 3, 9, 3)])
def test_host_engine_fermion_eval_one_pass_matches_oracle(engine, tmp_path, case):
    # fermion_eval: the amplitude, the local energies and the signed O rows in one pass over the
    # rows, against the oracle's amplitude, local energies and sums over every virtual
    # assignment (exact chi)
    from oracle import fermion as fm
    L1, L2, D, chi, n = case
    N = L1 * L2
    t_hop, U, mu = 1.0, 8.0, 4.0
    rng = np.random.default_rng(17 * L1 + 7 * L2 + D)
    T = fm.random_even_fpeps(L1, L2, D, rng, scale=0.5)
    for i, A in enumerate(fm.identity_fpeps(L1, L2)):
        T[i][(slice(None), 0, 0, 0, 0)] += A[:, 0, 0, 0, 0]
    S = rng.integers(0, 16, (n, N))
    for k in range(n):
        if sum(bin(int(x)).count("1") for x in S[k]) % 2:
            S[k, 0] ^= 1
    S = S.astype(np.uint8)
    lat = Lattice(L1, L2, D, J1=t_hop, J2=U)
    mu_bits = struct.unpack("<Q", struct.pack("<d", mu))[0]
    la, sg, es, ea, O = _run(engine, tmp_path, 7, lat, chi, _fermion_th64(T), S, seed=mu_bits)
    for k in range(n):
        grads, psi = fm.fpeps_log_derivative(L1, L2, T, S[k])
        assert sg[k] == np.sign(psi) and abs(la[k] - np.log(abs(psi))) <= 1e-10, k
        r_es, r_ea = fm.fpeps_local_energy(L1, L2, T, S[k], t_hop, U, mu)
        scale = max(1.0, abs(r_es), abs(r_ea))
        assert abs(es[k] - r_es) <= 1e-9 * scale and abs(ea[k] - r_ea) <= 1e-9 * scale, k
        ref = np.concatenate([g.ravel() for g in grads])
        assert np.max(np.abs(O[k] - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref))), k
