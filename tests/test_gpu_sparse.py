"""Block-sparse B from Schwarz screening (Section 2.1) on chain molecules, through the C ABI.

A screened AO pair is an exact zero in every B_P; the library then runs only the
nonzero K tiles of the first exchange GEMM and skips the zero chunks in rho and J.
Skipped terms are exact zeros, so K stays bit-exact against the oracle's emulation
of the same (screened) B, and J matches the oracle's FP64 J.
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


@pytest.fixture(scope="module")
def chain():
    """A 96-atom chain (nao 480, naux 1440) screened at 1e-12: 12 % of the AO pairs and 57 %
    of the first GEMM's K tiles survive."""
    mol = inputs.chain_molecule(96, 17)
    B = inputs.df_tensor(mol, 1e-12)
    return mol, B


@pytest.fixture(scope="module")
def short_chain():
    """A 60-atom chain (nao 300, naux 900) screened at 1e-12: 91 % of the K tiles survive."""
    mol = inputs.chain_molecule(60, 17)
    B = inputs.df_tensor(mol, 1e-12)
    return mol, B


def test_screened_chain_exchange_bitexact_vs_oracle(df, short_chain):
    """8 orbitals at 5 slices, the first GEMM in both layouts: CTA pairs with the (P, mu) rows
    on the MMA's M side (each pair runs the union of its two row tiles' K tiles) and single
    CTAs with the orbitals on M (the row tile's own K tiles): both bit-exact."""
    mol, B = short_chain
    C = inputs.orbitals(mol.nao, 8, 18)
    ref = O.emulated_exchange(B, C, 5)
    Bg = torch.from_numpy(B).cuda()
    Cg = torch.from_numpy(C).cuda()
    for pairs in (1, 0):
        ctx = df.Context(mol.nao, mol.naux, 8)
        ctx.set_cluster_pairs(pairs)
        ctx.setup(Bg)
        fk, fc = ctx.sparsity()
        assert fk < 0.95 and fc < 0.6
        assert np.array_equal(ctx.build_K(Cg, 5)[0].cpu().numpy(), ref)


@pytest.mark.parametrize("nocc", [60, 150])
def test_screened_chain_sparse_equals_dense(df, chain, nocc):
    """The block-sparse build equals the dense build of the same B bit for bit (skipped terms
    are exact zeros), in both first-GEMM layouts; 8 slices within 1e-10 of the oracle's K."""
    mol, B = chain
    C = inputs.orbitals(mol.nao, nocc, 21)
    Bg = torch.from_numpy(B).cuda()
    Cg = torch.from_numpy(C).cuda()
    ctx = df.Context(mol.nao, mol.naux, nocc)
    ctx.setup(Bg)
    fk, fc = ctx.sparsity()
    assert fk < 0.7 and fc < 0.5
    for s in (3, 5):
        Ks = ctx.build_K(Cg, s)[0].clone()
        ctx.set_sparse(False)
        Kd = ctx.build_K(Cg, s)[0].clone()
        ctx.set_sparse(True)
        assert torch.equal(Ks, Kd)
    K8 = ctx.build_K(Cg, 8)[0].cpu().numpy()
    K_ref = O.exchange(B, C)
    assert np.max(np.abs(K8 - K_ref)) <= 1e-10 * np.max(np.abs(K_ref))


def test_screened_chain_coulomb_vs_oracle(df, chain):
    mol, B = chain
    C = inputs.orbitals(mol.nao, 60, 19)
    D = inputs.density(C)
    ctx = df.Context(mol.nao, mol.naux, 60)
    Bg = torch.from_numpy(B).cuda()
    ctx.setup(Bg)
    J, rho = ctx.build_J(torch.from_numpy(D).cuda())
    J, rho = J.cpu().numpy(), rho.cpu().numpy()
    rho_ref = O.rho(B, D)
    J_ref = O.coulomb(B, rho_ref)
    assert np.max(np.abs(rho - rho_ref)) <= 1e-12 * np.max(np.abs(rho_ref))
    assert np.max(np.abs(J - J_ref)) <= 1e-12 * np.max(np.abs(J_ref))
    keep = inputs.schwarz_pairs(mol, 1e-12)
    assert np.all(J[~keep] == 0.0) and np.array_equal(J, J.T)
    ctx.set_sparse(False)
    Jd = ctx.build_J(torch.from_numpy(D).cuda())[0].cpu().numpy()
    assert np.array_equal(J, Jd)      # J's per-element sums are the dense ones; screened pairs 0


def test_dense_molecule_keeps_the_dense_path(df):
    """The cube molecule has no zero chunk: both fractions are 1 (no masks are used)."""
    mol, B, C, D = inputs.make_inputs(inputs.SMALL)
    ctx = df.Context(mol.nao, mol.naux, C.shape[1])
    Bg = torch.from_numpy(B).cuda()
    ctx.setup(Bg)
    assert ctx.sparsity() == (1.0, 1.0)


def test_screened_chain_in_a_batch(df, chain):
    """A batch mixing the screened chain and a dense molecule: grouped launches use each
    molecule's own masks; results equal the single builds."""
    s = 5
    mol, B = chain
    mols = [(B, inputs.orbitals(mol.nao, 60, 20))]
    m2, B2, C2, _ = inputs.make_inputs(inputs.SMALL)
    mols.append((B2, C2))
    ctxs, keep, Cs = [], [], []
    for Bm, Cm in mols:
        ctx = df.Context(Bm.shape[1], Bm.shape[0], Cm.shape[1], s_max=s)
        Bg = torch.from_numpy(Bm).cuda()
        ctx.setup(Bg)
        ctxs.append(ctx)
        keep.append(Bg)
        Cs.append(torch.from_numpy(Cm).cuda())
    single = [ctx.build_K(C, s)[0].clone() for ctx, C in zip(ctxs, Cs)]
    batch = df.Batch(ctxs)
    Ks = [torch.empty_like(k) for k in single]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.build_K(Cs, s, Ks)
    stream.synchronize()
    for k, k1 in zip(Ks, single):
        assert torch.equal(k, k1)
