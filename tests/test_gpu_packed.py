"""B given as packed upper triangles (df_setup_packed), through the C ABI.

The packed layout holds each B_P's upper triangle row by row, half the bytes of
the dense tensor (the symmetric storage Section 3.3 describes).  With the same
values, a packed context must give the dense context's results bit for bit:
the digit planes are the same, rho and J read the same values in the same
order, the FP64 comparison build runs the same per-P products, and the
sparsity masks of a screened B are the same.
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


def _pair(df, B, nocc, perm=None):
    naux, nao, _ = B.shape
    dense = df.Context(nao, naux, nocc)
    packed = df.Context(nao, naux, nocc)
    Bg = torch.from_numpy(B).cuda()
    Bp = torch.from_numpy(inputs.pack_upper(B)).cuda()
    assert Bp.shape == (naux, nao * (nao + 1) // 2)
    dense.setup(Bg, perm=perm)
    packed.setup_packed(Bp, perm=perm)
    return dense, packed, (Bg, Bp)


def test_packed_equals_dense_and_the_oracle(df):
    mol, B, C, D = inputs.make_inputs(inputs.SMALL)
    dense, packed, keep = _pair(df, B, C.shape[1])
    Cg, Dg = torch.from_numpy(C).cuda(), torch.from_numpy(D).cuda()
    for s in (3, 5):
        Kp = packed.build_K(Cg, s)[0].clone()
        assert torch.equal(Kp, dense.build_K(Cg, s)[0])
    assert np.array_equal(Kp.cpu().numpy(), O.emulated_exchange(B, C, 5))
    Jp, rp = packed.build_J(Dg)
    Jd, rd = dense.build_J(Dg)
    assert torch.equal(Jp, Jd) and torch.equal(rp, rd)
    K64p = packed.build_K(Cg, 0)[0].clone()
    K64d = dense.build_K(Cg, 0)[0]
    assert float((K64p - K64d).abs().max()) <= 1e-14 * float(K64d.abs().max())
    Fp = df.block_features(packed, C.shape[1], 1e-10, 1e-4, 1e-8, 5)
    Fd = df.block_features(dense, C.shape[1], 1e-10, 1e-4, 1e-8, 5)
    assert float((Fp - Fd).abs().max()) < 1e-6
    E = packed.energy(Dg, Jp, Kp, rp)
    EJ, EK = O.energies(D, O.coulomb(B, O.rho(B, D)), O.exchange(B, C))
    assert abs(E[0] - EJ) < 1e-9 and abs(E[1] - EJ) < 1e-9


def test_packed_in_magnitude_order(df):
    mol, B, C, D = inputs.make_inputs(inputs.SMALL)
    perm = np.argsort(-np.abs(B).reshape(B.shape[0], -1).max(1))
    dense, packed, keep = _pair(df, B, C.shape[1], perm=perm)
    Cg = torch.from_numpy(C).cuda()
    Kp = packed.build_K(Cg, 5)[0]
    assert torch.equal(Kp, dense.build_K(Cg, 5)[0])
    assert np.array_equal(Kp.cpu().numpy(), O.emulated_exchange(B[perm], C, 5))


def test_packed_screened_chain(df):
    """A screened 96-atom chain: the same masks, the same block-sparse K and J as dense."""
    mol = inputs.chain_molecule(96, 17)
    B = inputs.df_tensor(mol, 1e-12)
    C = inputs.orbitals(mol.nao, 60, 22)
    dense, packed, keep = _pair(df, B, 60)
    assert packed.sparsity() == dense.sparsity() and packed.sparsity()[0] < 0.7
    Cg, Dg = torch.from_numpy(C).cuda(), torch.from_numpy(inputs.density(C)).cuda()
    assert torch.equal(packed.build_K(Cg, 5)[0], dense.build_K(Cg, 5)[0])
    assert torch.equal(packed.build_J(Dg)[0], dense.build_J(Dg)[0])


def test_packed_in_a_batch(df):
    s = 5
    mols = [inputs.make_inputs(inputs.SMALL)]
    m2 = inputs.molecule(30, 51)
    B2 = inputs.df_tensor(m2)
    mols.append((m2, B2, inputs.orbitals(m2.nao, 30, 52), None))
    ctxs, keep, Cs, Ds = [], [], [], []
    for mol, B, C, _ in mols:
        ctx = df.Context(B.shape[1], B.shape[0], C.shape[1], s_max=s)
        Bp = torch.from_numpy(inputs.pack_upper(B)).cuda()
        ctx.setup_packed(Bp)
        ctxs.append(ctx)
        keep.append(Bp)
        Cs.append(torch.from_numpy(C).cuda())
        Ds.append(torch.from_numpy(inputs.density(C)).cuda())
    single = [ctx.build_K(C, s)[0].clone() for ctx, C in zip(ctxs, Cs)]
    singleJ = [ctx.build_J(D)[0].clone() for ctx, D in zip(ctxs, Ds)]
    batch = df.Batch(ctxs)
    Ks = [torch.empty_like(k) for k in single]
    Js = [torch.empty_like(j) for j in singleJ]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.build_K(Cs, s, Ks)
        batch.build_J(Ds, Js)
    stream.synchronize()
    for k, k1 in zip(Ks, single):
        assert torch.equal(k, k1)
    for j, j1 in zip(Js, singleJ):
        assert torch.equal(j, j1)
