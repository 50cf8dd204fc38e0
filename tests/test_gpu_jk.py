"""The Coulomb and exchange builds in one call (df_build_JK), through the C ABI.

df_build_JK forks rho and J onto an internal high-priority stream after the
first exchange GEMM, so that these FP64-pipe-bound kernels share the SMs with
the X split.  Its J, rho and K must equal those of df_build_J followed by
df_build_K bit for bit, for every overlap setting, on a dense and a packed B
(and on a Schwarz-screened one, which runs the two builds in order), at fixed
and adaptive slice counts, over consecutive calls on a side stream; and they
must match the CPU oracle (K bit-exact against the oracle's emulation at 5
slices, J within the FP64 summation bound, energies within 1e-9 Eh).
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
def small():
    mol, B, C, D = inputs.make_inputs(inputs.SMALL)
    return B, C, D


def _separate(ctx, Dg, Cg, s):
    J, rho = ctx.build_J(Dg)
    K, st = ctx.build_K(Cg, s)
    return J.clone(), rho.clone(), K.clone(), st


def _same(a, b):
    return all(torch.equal(x, y) for x, y in zip(a[:3], b[:3]))


def test_jk_equals_separate_builds_and_oracle(df, small):
    B, C, D = small
    ctx = df.Context(B.shape[1], B.shape[0], C.shape[1])
    Bg = torch.from_numpy(B).cuda()
    ctx.setup(Bg)
    Cg, Dg = torch.from_numpy(C).cuda(), torch.from_numpy(D).cuda()
    ref = _separate(ctx, Dg, Cg, 5)
    for ctas in (0, 1, 2, 4):
        ctx.set_jk_overlap(ctas)
        got = ctx.build_JK(Dg, Cg, 5)
        assert _same(got, ref), ctas
        assert list(got[3].slices[:ctx.nblk]) == [5] * ctx.nblk
    J, rho, K, _ = got
    assert np.array_equal(K.cpu().numpy(), O.emulated_exchange(B, C, 5))
    rho_ref = O.rho(B, D)
    J_ref = O.coulomb(B, rho_ref)
    assert float(np.abs(J.cpu().numpy() - J_ref).max()) <= 1e-12 * float(np.abs(J_ref).max())
    EJ, EJ2, EK = ctx.energy(Dg, J, K, rho)
    EJ_ref, EK_ref = O.energies(D, J_ref, O.exchange(B, C))
    assert abs(EJ - EJ_ref) <= 1e-9 and abs(EJ2 - EJ_ref) <= 1e-9 and abs(EK - EK_ref) <= 1e-9


def test_jk_adaptive_and_native_counts(df, small):
    """-1 takes the current level's count (level 4: 3 slices) as df_build_K does; 0 (native
    FP64) runs the two builds in order."""
    B, C, D = small
    ctx = df.Context(B.shape[1], B.shape[0], C.shape[1])
    ctx.setup(torch.from_numpy(B).cuda())
    Cg, Dg = torch.from_numpy(C).cuda(), torch.from_numpy(D).cuda()
    ctx.adaptive_reset()
    ref = _separate(ctx, Dg, Cg, df.ADAPTIVE)
    got = ctx.build_JK(Dg, Cg, df.ADAPTIVE)
    assert _same(got, ref)
    assert got[3].level == 4 and list(got[3].slices[:ctx.nblk]) == [3] * ctx.nblk
    ref64 = _separate(ctx, Dg, Cg, 0)
    got64 = ctx.build_JK(Dg, Cg, 0)
    assert torch.equal(got64[0], ref64[0]) and torch.equal(got64[1], ref64[1])
    assert float((got64[2] - ref64[2]).abs().max()) <= 1e-14 * float(ref64[2].abs().max())


def test_jk_consecutive_calls_on_a_side_stream(df):
    """Two builds with different densities back to back on a non-default stream (the work
    counters are reset per call, the second call's Coulomb kernels wait for the first's
    exchange), on a molecule whose rho and J take many items per CTA (naux 1800, nao 600)."""
    mol, B, C, D = inputs.make_inputs(inputs.MEDIUM)
    ctx = df.Context(mol.nao, mol.naux, C.shape[1])
    Bg = torch.from_numpy(B).cuda()
    ctx.setup(Bg)
    C2 = inputs.orbitals(mol.nao, C.shape[1], 91)
    D2 = inputs.density(C2)
    pairs = [(torch.from_numpy(D).cuda(), torch.from_numpy(C).cuda()),
             (torch.from_numpy(D2).cuda(), torch.from_numpy(C2).cuda())]
    refs = [_separate(ctx, Dg, Cg, 5) for Dg, Cg in pairs]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        outs = [ctx.build_JK(Dg, Cg, 5, stream=side) for Dg, Cg in pairs]
    side.synchronize()
    for got, ref in zip(outs, refs):
        assert _same(got, ref)
    assert not torch.equal(outs[0][0], outs[1][0])


def test_jk_packed_and_screened(df):
    """A Schwarz-screened chain, dense (zero chunks skipped in rho, J and the first GEMM; the
    builds run in order) and packed with the sparse kernels off (the Coulomb build beside the X
    split), gives the separate builds' results; K of the chain is bit-exact against the oracle."""
    mol = inputs.chain_molecule(60, 17)
    B = inputs.df_tensor(mol, 1e-12)
    C = inputs.orbitals(mol.nao, 8, 18)
    D = inputs.density(C)
    Cg, Dg = torch.from_numpy(C).cuda(), torch.from_numpy(D).cuda()
    Bg = torch.from_numpy(B).cuda()
    Bp = torch.from_numpy(inputs.pack_upper(B)).cuda()
    dense = df.Context(mol.nao, mol.naux, 8)
    dense.setup(Bg)
    packed = df.Context(mol.nao, mol.naux, 8)
    packed.setup_packed(Bp)
    packed.set_sparse(False)
    assert dense.sparsity()[1] < 0.95
    results = []
    for ctx in (dense, packed):
        ref = _separate(ctx, Dg, Cg, 5)
        got = ctx.build_JK(Dg, Cg, 5)
        assert _same(got, ref)
        results.append(got)
    assert _same(results[0], results[1])
    assert np.array_equal(results[0][2].cpu().numpy(), O.emulated_exchange(B, C, 5))


def test_jk_argument_errors(df, small):
    B, C, D = small
    ctx = df.Context(B.shape[1], B.shape[0], C.shape[1])
    Cg, Dg = torch.from_numpy(C).cuda(), torch.from_numpy(D).cuda()
    with pytest.raises(df.DFError) as e:
        ctx.build_JK(Dg, Cg, 5)  # before setup
    assert e.value.status == -7
    ctx.setup(torch.from_numpy(B).cuda())
    with pytest.raises(df.DFError) as e:
        ctx.build_JK(Dg, Cg, 9)
    assert e.value.status == -1
    with pytest.raises(df.DFError) as e:
        ctx.set_jk_overlap(5)
    assert e.value.status == -1
