"""Pins of the SCF oracle (one-electron integrals, RHF loop) and parity of the
input generator's one-electron integrals with it."""
import math

import numpy as np
import pytest

from oracle import df_oracle as O
from oracle import scf_oracle as SO
from paper_2601_08077_gb300 import inputs


def test_one_function_closed_forms():
    a, Z = 0.7, 2.0
    x = np.zeros((1, 3))
    e = np.array([a])
    assert SO.overlap(x, e)[0, 0] == pytest.approx(1.0, abs=1e-15)
    assert SO.kinetic(x, e)[0, 0] == pytest.approx(1.5 * a, rel=1e-14)
    # <1/r> of a normalised s Gaussian is 2 sqrt(2a/pi)
    assert SO.nuclear(x, e, x, [Z])[0, 0] == pytest.approx(-Z * 2.0 * math.sqrt(2.0 * a / math.pi), rel=1e-14)


def test_two_centre_overlap_and_kinetic_closed_forms():
    a, b, R = 0.8, 1.3, 1.7
    x = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, R]])
    e = np.array([a, b])
    p, mu = a + b, a * b / (a + b)
    s_ab = (4.0 * a * b / p ** 2) ** 0.75 * math.exp(-mu * R * R)
    assert SO.overlap(x, e)[0, 1] == pytest.approx(s_ab, rel=1e-14)
    assert SO.kinetic(x, e)[0, 1] == pytest.approx(mu * (3 - 2 * mu * R * R) * s_ab, rel=1e-13)


def test_matrices_symmetric_and_definite():
    mol = inputs.molecule(8, 5)
    Z = inputs.nuclear_charges(mol)
    S = SO.overlap(mol.ao_xyz, mol.ao_exp)
    T = SO.kinetic(mol.ao_xyz, mol.ao_exp)
    V = SO.nuclear(mol.ao_xyz, mol.ao_exp, mol.xyz, Z)
    for M in (S, T, V):
        assert np.array_equal(M, M.T)
    assert np.linalg.eigvalsh(S)[0] > 0 and np.linalg.eigvalsh(T)[0] > 0
    assert np.linalg.eigvalsh(V)[-1] < 0                      # attraction
    assert SO.nuclear_repulsion(np.array([[0, 0, 0.0], [0, 0, 2.0]]), [2.0, 3.0]) == pytest.approx(3.0)


def test_generator_matches_oracle():
    mol = inputs.molecule(20, 0)
    Z = inputs.nuclear_charges(mol)
    S, T, V, En = inputs.one_electron(mol, Z)
    np.testing.assert_allclose(S, SO.overlap(mol.ao_xyz, mol.ao_exp), rtol=0, atol=1e-14)
    np.testing.assert_allclose(T, SO.kinetic(mol.ao_xyz, mol.ao_exp), rtol=0, atol=1e-13)
    np.testing.assert_allclose(V, SO.nuclear(mol.ao_xyz, mol.ao_exp, mol.xyz, Z), rtol=0, atol=1e-13)
    assert En == pytest.approx(SO.nuclear_repulsion(mol.xyz, Z), rel=1e-14)


def test_scf_one_function_helium_is_closed_form():
    # one normalised s function on a He nucleus; the single auxiliary function
    # exp(-2a r^2) fits the product density exactly, so DF-J = DF-K = (aa|aa)
    # and E = 2 h + (aa|aa) with (aa|aa) = 2 sqrt(a/pi)
    a, Z = 0.9, 2.0
    x = np.zeros((1, 3))
    e = np.array([a])
    h = SO.kinetic(x, e) + SO.nuclear(x, e, x, [Z])
    B = O.df_tensor(O.int3c(x, e, x, np.array([2.0 * a])), O.metric(x, np.array([2.0 * a])))
    res = SO.scf(h, SO.overlap(x, e), 1, SO.df_jk(B))
    assert res["converged"]
    assert res["E"] == pytest.approx(2.0 * h[0, 0] + 2.0 * math.sqrt(a / math.pi), rel=1e-13)


def test_scf_converges_and_is_stationary():
    mol, B, C, D = inputs.make_inputs(inputs.SMALL)
    Z = inputs.nuclear_charges(mol)
    S = SO.overlap(mol.ao_xyz, mol.ao_exp)
    h = SO.kinetic(mol.ao_xyz, mol.ao_exp) + SO.nuclear(mol.ao_xyz, mol.ao_exp, mol.xyz, Z)
    res = SO.scf(h, S, mol.n_atoms, SO.df_jk(B), SO.nuclear_repulsion(mol.xyz, Z))
    assert res["converged"]
    F, Dm = res["F"], res["D"]
    assert np.max(np.abs(F @ Dm @ S - S @ Dm @ F)) < 1e-6        # commutes at convergence
    assert np.allclose(Dm @ S @ Dm, 2.0 * Dm, atol=1e-10)          # idempotent (D S D = 2 D)
    assert abs(np.sum(Dm * S) - 2 * mol.n_atoms) < 1e-9            # electron count
    assert res["E"] < res["history"][0]


def test_scf_energy_is_invariant_to_the_order_of_atoms_and_aux_functions():
    # relabelling basis functions (atom order) and auxiliary functions changes
    # every matrix but not the physics: a dropped term or a transposed index
    # in the Fock build would break this
    mol, B, C, D = inputs.make_inputs(inputs.SMALL)
    Z = inputs.nuclear_charges(mol)
    S = SO.overlap(mol.ao_xyz, mol.ao_exp)
    h = SO.kinetic(mol.ao_xyz, mol.ao_exp) + SO.nuclear(mol.ao_xyz, mol.ao_exp, mol.xyz, Z)
    En = SO.nuclear_repulsion(mol.xyz, Z)
    ref = SO.scf(h, S, mol.n_atoms, SO.df_jk(B), En)
    rng = np.random.default_rng(5)
    p = rng.permutation(mol.nao)
    q = rng.permutation(B.shape[0])
    Bp = np.ascontiguousarray(B[q][:, p][:, :, p])
    res = SO.scf(h[np.ix_(p, p)], S[np.ix_(p, p)], mol.n_atoms, SO.df_jk(Bp), En)
    assert res["converged"] and ref["converged"]
    assert abs(res["E"] - ref["E"]) < 1e-9
