"""rho and J at the shapes that stress their work split, through the C ABI.

rho streams the strictly upper elements of each B_P in row-pair order (pair q
is row q followed by row nao-1-q; for odd nao the middle row comes last
alone), thread t of a CTA taking elements t, t + 256, ...; J takes its
elements in chunks of a row pair.  Odd nao (the lone middle row), nao below
the CTA's 256 threads (a thread's next element lies several pairs ahead),
nao = 1, 2 and 3 (the Coulomb build alone), and a naux that is not a
multiple of J's eight loads in flight: rho and J against the oracle's
definitions within the FP64 summation bound, dense and packed layouts equal to
each other bit for bit, and df_build_JK's short grids (items taken from a
counter) equal to df_build_J's full grids bit for bit.
"""
import numpy as np
import pytest
import torch

from oracle import df_oracle as O
from paper_2601_08077_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def df():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_08077_gb300 import build, df as dfmod
    build.build_all()
    return dfmod


def _random(seed, naux, nao, nocc):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((naux, nao, nao))
    B = 0.5 * (B + B.transpose(0, 2, 1))
    C = np.linalg.qr(rng.standard_normal((nao, nao)))[0][:, :nocc] if nocc <= nao else None
    return B, np.ascontiguousarray(C)


def _check(df, B, C, jk=True):
    naux, nao, _ = B.shape
    nocc = C.shape[1]
    D = inputs.density(C)
    rho_ref = O.rho(B, D)
    J_ref = O.coulomb(B, rho_ref)
    # FP64 reordering bounds of the sums (both sides' roundings): rho_P sums nao^2 terms of size
    # |B||D|; J_mn sums naux terms of size |B||rho|, plus |B| times rho's own error per term
    eps, bmax = np.finfo(float).eps, np.max(np.abs(B))
    tol_rho = 4 * nao * nao * eps * bmax * np.max(np.abs(D))
    tol_J = 4 * naux * eps * bmax * np.max(np.abs(rho_ref)) + naux * bmax * tol_rho
    Dg, Cg = torch.from_numpy(D).cuda(), torch.from_numpy(C).cuda()
    Bg = torch.from_numpy(B).cuda()
    Bp = torch.from_numpy(inputs.pack_upper(B)).cuda()
    out = []
    for packed in (False, True):
        ctx = df.Context(nao, naux, nocc)
        if packed:
            ctx.setup_packed(Bp)
        else:
            ctx.setup(Bg)
        J, rho = ctx.build_J(Dg)
        J, rho = J.clone(), rho.clone()
        if jk:
            J2, rho2, _, _ = ctx.build_JK(Dg, Cg, 5)
            assert torch.equal(J, J2) and torch.equal(rho, rho2)
        ctx.sync_status()
        out.append((J.cpu().numpy(), rho.cpu().numpy()))
    (Jd, rd), (Jp, rp) = out
    assert np.array_equal(Jd, Jp) and np.array_equal(rd, rp)
    assert np.max(np.abs(rd - rho_ref)) <= tol_rho
    assert np.max(np.abs(Jd - J_ref)) <= tol_J
    assert np.array_equal(Jd, Jd.T)


@pytest.mark.parametrize("nao, naux", [(33, 29), (255, 13), (257, 11)])
def test_coulomb_random_shapes(df, nao, naux):
    B, C = _random(500 + nao, naux, nao, 1)
    _check(df, B, C)


@pytest.mark.parametrize("nao, naux", [(1, 5), (2, 3), (3, 7)])
def test_coulomb_tiny(df, nao, naux):
    """No or one or three off-diagonal elements per B_P (the Coulomb build alone: an exchange
    build of a 1-3 function basis is not a case the slice GEMM's tiles are meant for)."""
    B, C = _random(600 + nao, naux, nao, 1)
    _check(df, B, C, jk=False)


def test_coulomb_odd_molecule(df):
    """27 atoms: nao 135 (odd), naux 405 (a ragged fourth block of 21 functions)."""
    mol, B, C, D = inputs.make_inputs(inputs.Workload("df-27atom-nao135-naux405-nocc27", 27, 27, 7300))
    _check(df, B, C)
