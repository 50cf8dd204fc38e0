"""Host-side parts of the GPU SCF driver (orthogonaliser, DIIS) on CPU tensors,
against the oracle's restatements."""
import numpy as np
import torch

from oracle import scf_oracle as SO
from paper_2601_08077_gb300 import inputs, scf


def test_orthogonaliser_matches_oracle_and_whitens():
    mol = inputs.molecule(8, 5)
    S = SO.overlap(mol.ao_xyz, mol.ao_exp)
    X = scf._orthogonaliser(torch.from_numpy(S)).numpy()
    Xo = SO.orthogonaliser(S)
    assert X.shape == Xo.shape
    np.testing.assert_allclose(X.T @ S @ X, np.eye(X.shape[1]), atol=1e-10)
    # the same subspace: X Xo^T S projects onto it either way
    np.testing.assert_allclose(X @ X.T, Xo @ Xo.T, atol=1e-8)


def test_diis_matches_oracle():
    rng = np.random.default_rng(2)
    Fs = [rng.standard_normal((6, 6)) for _ in range(4)]
    Fs = [0.5 * (F + F.T) for F in Fs]
    errs = [rng.standard_normal((6, 6)) * 10.0 ** -k for k in range(4)]
    ref = SO.diis_extrapolate(Fs, errs)
    got = scf._diis([torch.from_numpy(F) for F in Fs], [torch.from_numpy(e) for e in errs]).numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12)


def test_diis_is_affine_and_exact_on_a_zero_residual():
    # coefficients sum to one: a history of identical F returns it; a zero
    # error vector gets all the weight
    F = torch.eye(4, dtype=torch.float64) * 3.0
    e = [torch.randn(4, 4, dtype=torch.float64) for _ in range(3)]
    assert torch.allclose(scf._diis([F, F, F], e), F)
    e0 = [torch.ones(4, 4, dtype=torch.float64), torch.zeros(4, 4, dtype=torch.float64)]
    G = torch.full((4, 4), 7.0, dtype=torch.float64)
    assert torch.allclose(scf._diis([F, G], e0), G)
