"""Fermionic PEPS amplitudes on the GPU (peps_famp_*; Sec. II fermionic vectorisation, Fig. 1b,
Sec. III.B) through the C ABI against the oracle: random parity-even PEPS (exact chi) in
FP64 to 1e-10 in log|psi| with the sign, near-product states in FP32 and TF32, odd
configurations, invalid entries, and a PEPS carrying hopping gates against the
Jordan-Wigner state vector."""
import numpy as np
import pytest

from oracle import fermion as fm
from paper_2409_05285_gb300 import binding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_05285_gb300.build import build
    build()


def _flat(T):
    return np.concatenate([t.ravel() for t in T])


def _even_configs(N, n, rng):
    S = rng.integers(0, 16, (n, N)).astype(np.uint8)
    for k in range(n):
        if sum(bin(int(x)).count("1") for x in S[k]) % 2:
            S[k, 0] ^= 1            # flip one occupation: even total parity
    return S


def _near_product(nr, nc, D, rng, noise):
    # |I>'s tensors in the first (even) virtual slot plus an even random perturbation
    T = fm.random_even_fpeps(nr, nc, D, rng, scale=noise)
    for i, A in enumerate(fm.identity_fpeps(nr, nc)):
        T[i][(slice(None), 0, 0, 0, 0)] += A[:, 0, 0, 0, 0]
    return T


@pytest.mark.parametrize("shape", [(2, 2, 2, 8), (3, 3, 2, 8), (4, 4, 2, 16), (3, 4, 3, 16)])
def test_fp64_amplitudes_match_oracle(shape):
    nr, nc, D, chi = shape
    rng = np.random.default_rng(nr * 100 + nc * 10 + D)
    T = fm.random_even_fpeps(nr, nc, D, rng)
    S = _even_configs(nr * nc, 24, rng)
    f = binding.FermionAmplitudes(nr, nc, D, chi, 24, precision=binding.PEPS_FP64)
    la, sg = f.eval(_flat(T), S)
    for k in range(len(S)):
        ref = fm.fpeps_amplitude_bosonic(nr, nc, T, S[k])
        assert ref != 0.0
        assert sg[k] == np.sign(ref), k
        assert abs(la[k] - np.log(abs(ref))) <= 1e-10, k
    f.close()


@pytest.mark.parametrize("prec,tol", [(binding.PEPS_FP32, 2e-4), (binding.PEPS_TF32, 5e-2)])
def test_float_amplitudes_on_near_product_states(prec, tol):
    nr, nc, D, chi = 3, 3, 2, 8
    rng = np.random.default_rng(5)
    T = _near_product(nr, nc, D, rng, 0.1)
    # configurations on the support of |I> (system and ancilla occupations equal) and random
    ident = rng.integers(0, 4, (16, nr * nc))
    S = np.concatenate([(ident | (ident << 2)).astype(np.uint8), _even_configs(nr * nc, 16, rng)])
    f = binding.FermionAmplitudes(nr, nc, D, chi, len(S), precision=prec)
    la, sg = f.eval(_flat(T), S)
    for k in range(16):          # the |I> support: amplitudes of order one
        ref = fm.fpeps_amplitude_bosonic(nr, nc, T, S[k])
        assert sg[k] == np.sign(ref), k
        assert abs(la[k] - np.log(abs(ref))) <= tol, k
    f.close()


def test_odd_and_invalid_configurations():
    nr, nc, D, chi = 3, 3, 2, 8
    rng = np.random.default_rng(9)
    T = fm.random_even_fpeps(nr, nc, D, rng)
    S = _even_configs(nr * nc, 4, rng)
    S[1, 2] ^= 1                 # odd total parity: psi = 0
    f = binding.FermionAmplitudes(nr, nc, D, chi, 4, precision=binding.PEPS_FP64)
    la, sg = f.eval(_flat(T), S)
    assert sg[1] == 0 and np.isneginf(la[1])
    assert sg[0] != 0 and np.isfinite(la[0])
    S[2, 0] = 16
    with pytest.raises(binding.PepsError) as e:
        f.eval(_flat(T), S)
    assert e.value.code == binding.PEPS_EINVAL
    with pytest.raises(binding.PepsError):
        f.eval(_flat(T)[:-1], S)
    f.close()


def test_gated_identity_against_the_fermionic_state():
    # hopping gates of Eq. 14 (spin up: four factors, bond dimension 4) on the two crossing
    # vertical bonds of 2x2, applied to |I>: the GPU's amplitudes on the state's support
    # equal the Jordan-Wigner state vector's
    nr, nc = 2, 2
    fac = fm.hopping_gate_factors(1.0, 0.3, spins=(0,))
    T = fm.identity_fpeps(nr, nc)
    for (i, j, kind) in [(0, 2, "v"), (1, 3, "v")]:
        T = fm.apply_gate_to_product(T, i, j, kind, fac)
    # pad every site to one bond dimension (the unused legs stay of dimension one)
    psi = fm.fpeps_state(nr, nc, T)
    support = np.nonzero(np.abs(psi) > 1e-10 * np.max(np.abs(psi)))[0]
    S = np.array([fm.local_indices(int(st), nr * nc) for st in support], dtype=np.uint8)
    D = max(max(t.shape[1:]) for t in T)
    Tp = []
    for r in range(nr):
        for c in range(nc):
            t = T[r * nc + c]
            dims = (1 if c == 0 else D, 1 if c == nc - 1 else D, 1 if r == 0 else D, 1 if r == nr - 1 else D)
            A = np.zeros((16,) + dims)
            A[(slice(None),) + tuple(slice(0, x) for x in t.shape[1:])] = t
            Tp.append(A)
    f = binding.FermionAmplitudes(nr, nc, D, 16, len(S), precision=binding.PEPS_FP64)
    la, sg = f.eval(_flat(Tp), S)
    ref = psi[support]
    assert np.array_equal(sg, np.sign(ref).astype(np.int8))
    assert np.max(np.abs(la - np.log(np.abs(ref)))) <= 1e-10
    f.close()


@pytest.mark.parametrize("prec,tol", [(binding.PEPS_FP64, 1e-9), (binding.PEPS_FP32, 1e-3)])
def test_local_energies_match_oracle(prec, tol):
    # E_sys and E_anc (Eq. 9, terms of Eq. 14 with Jordan-Wigner signs) against the oracle's
    # row-contracted ratios, on a near-product state of 3x3 at exact chi
    nr, nc, D, chi, t_hop, U, mu = 3, 3, 2, 8, 1.0, 8.0, 4.0
    rng = np.random.default_rng(21)
    T = _near_product(nr, nc, D, rng, 0.3)
    ident = rng.integers(0, 4, (6, nr * nc))
    S = np.concatenate([(ident | (ident << 2)).astype(np.uint8), _even_configs(nr * nc, 6, rng)])
    f = binding.FermionAmplitudes(nr, nc, D, chi, len(S), precision=prec)
    la, sg, es, ea = f.local_energy(_flat(T), S, t_hop, U, mu)
    for k in range(len(S)):
        r_es, r_ea = fm.fpeps_local_energy(nr, nc, T, S[k], t_hop, U, mu)
        scale = max(1.0, abs(r_es), abs(r_ea))
        assert abs(es[k] - r_es) <= tol * scale, k
        assert abs(ea[k] - r_ea) <= tol * scale, k
    f.close()


def test_local_energies_of_the_gated_state_estimate_its_energy():
    # the gated 2x2 state of the test above: the |psi|^2-weighted average of (E_sys + E_anc)/2
    # over its whole support is its energy <H(c)> (Eq. 11 estimator, exact enumeration)
    nr, nc, t_hop, U, mu = 2, 2, 1.0, 8.0, 4.0
    fac = fm.hopping_gate_factors(1.0, 0.3, spins=(0,))
    T = fm.identity_fpeps(nr, nc)
    for (i, j, kind) in [(0, 2, "v"), (1, 3, "v")]:
        T = fm.apply_gate_to_product(T, i, j, kind, fac)
    psi = fm.fpeps_state(nr, nc, T)
    support = np.nonzero(np.abs(psi) > 1e-12 * np.max(np.abs(psi)))[0]
    S = np.array([fm.local_indices(int(st), nr * nc) for st in support], dtype=np.uint8)
    D = max(max(t.shape[1:]) for t in T)
    Tp = []
    for r in range(nr):
        for c in range(nc):
            t = T[r * nc + c]
            dims = (1 if c == 0 else D, 1 if c == nc - 1 else D, 1 if r == 0 else D, 1 if r == nr - 1 else D)
            A = np.zeros((16,) + dims)
            A[(slice(None),) + tuple(slice(0, x) for x in t.shape[1:])] = t
            Tp.append(A)
    f = binding.FermionAmplitudes(nr, nc, D, 16, len(S), precision=binding.PEPS_FP64)
    la, sg, es, ea = f.local_energy(_flat(Tp), S, t_hop, U, mu)
    w = np.exp(2 * (la - la.max()))
    E = np.sum(w * 0.5 * (es + ea)) / np.sum(w) / (nr * nc)
    E_ref, _ = fm.observables(nr, nc, t_hop, U, mu, psi)
    assert E == pytest.approx(E_ref, rel=1e-10)
    f.close()


@pytest.mark.parametrize("prec,tol", [(binding.PEPS_FP64, 1e-9), (binding.PEPS_FP32, 1e-3)])
def test_log_derivatives_match_oracle(prec, tol):
    # O (Eq. 8) of a random even PEPS (3x3, exact chi) against the oracle's sum over virtual
    # assignments, entry by entry in the layout [site][dl][dr][du][dd]
    nr, nc, D, chi = 3, 3, 2, 8
    rng = np.random.default_rng(33)
    T = fm.random_even_fpeps(nr, nc, D, rng, scale=0.5)
    S = _even_configs(nr * nc, 4, rng)
    f = binding.FermionAmplitudes(nr, nc, D, chi, 4, precision=prec)
    O = f.log_derivative(_flat(T), S).astype(np.float64)
    for k in range(len(S)):
        grads, _ = fm.fpeps_log_derivative(nr, nc, T, S[k])
        ref = np.concatenate([g.ravel() for g in grads])
        scale = max(1.0, np.max(np.abs(ref)))
        assert np.max(np.abs(O[k] - ref)) <= tol * scale, k
    f.close()


@pytest.mark.parametrize("prec,tol", [(binding.PEPS_FP64, 1e-10), (binding.PEPS_TF32, 5e-2)])
def test_bench_size_amplitudes_match_oracle(prec, tol):
    # the fermion bench's configuration (6x6, D = 4, chi = 16, 1024 chains, its perturbed |I>
    # from peps_famp_init_theta): six sampled configurations, on and one hop off the |I>
    # support, against the oracle's exact row-vector contraction.  chi = 16 truncates here;
    # on this state the truncated contraction differs from the exact one by under 1e-14 in
    # log|psi| (measured with the host build of the engine), so FP64 is held to 1e-10.
    from oracle import fermion_vmc as fv
    from paper_2409_05285_gb300 import workloads as wl
    L, D, chi, n = 6, 4, 16, 1024
    th = binding.famp_init_theta(L, L, D, 1e-3, 0)
    T = fv.unflatten(th, [np.zeros((16,) + d) for d in wl.site_dims(L, L, D)])
    S = wl.fermion_support_configs(n, L * L, 1)
    for k in range(3, 6):
        x = fv.propose(list(S[k]), ("hop", 0, 1, 0)) or fv.propose(list(S[k]), ("hop", 0, 1, 1))
        if x:
            S[k] = x
    f = binding.FermionAmplitudes(L, L, D, chi, n, precision=prec)
    la, sg = f.eval(th, S)
    amp = fm.fpeps_amplitude_function(L, L, T)
    for k in range(6):
        ref = amp(S[k])
        assert sg[k] == np.sign(ref), k
        assert abs(la[k] - np.log(abs(ref))) <= tol, k
    assert np.all(sg != 0)
    f.close()
