"""Batched builds: grouped persistent launches over molecules of uneven size, graph capture, autotuner."""
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
def molecules():
    out = []
    for atoms, seed in [(20, 11), (31, 12), (25, 13), (12, 14)]:
        mol = inputs.molecule(atoms, seed)
        B = inputs.df_tensor(mol)
        C = inputs.orbitals(mol.nao, atoms, seed + 1)
        out.append((B, C, inputs.density(C)))
    return out


def test_batch_matches_single_builds_and_oracle(df, molecules):
    s = 5
    ctxs, keep = [], []
    for B, C, D in molecules:
        ctx = df.Context(B.shape[1], B.shape[0], C.shape[1], s_max=s)
        Bg = torch.from_numpy(B).cuda()
        ctx.setup(Bg)
        ctxs.append(ctx)
        keep.append(Bg)
    Cs = [torch.from_numpy(C).cuda() for _, C, _ in molecules]
    Ds = [torch.from_numpy(D).cuda() for _, _, D in molecules]
    single = [ctx.build_K(C, s)[0].clone() for ctx, C in zip(ctxs, Cs)]
    Js1 = [ctx.build_J(D)[0].clone() for ctx, D in zip(ctxs, Ds)]
    batch = df.Batch(ctxs)
    Ks = [torch.full_like(k, float("nan")) for k in single]
    Js = [torch.full_like(j, float("nan")) for j in Js1]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.build_K(Cs, s, Ks)          # captures the graph
        batch.build_J(Ds, Js)
        for k in Ks:
            k.fill_(float("nan"))
        batch.build_K(Cs, s, Ks)          # replays it
    stream.synchronize()
    for k, k1 in zip(Ks, single):
        assert torch.equal(k, k1)
    for j, j1 in zip(Js, Js1):
        assert torch.equal(j, j1)
    B, C, D = molecules[1]
    assert np.array_equal(Ks[1].cpu().numpy(), O.emulated_exchange(B, C, s))
    choice = batch.autotune(Cs, s, Ks)
    assert choice[0] in (1, 2, 4, 8) and choice[1] in (0, 1) and choice[2] in (0, 1)
    with torch.cuda.stream(stream):
        for k in Ks:
            k.fill_(0.0)
        batch.build_K(Cs, s, Ks)
    stream.synchronize()
    for k, k1 in zip(Ks, single):
        assert torch.equal(k, k1)


def test_autotuner_choice_depends_on_the_molecule_mix(df):
    """Two seeded mixes from the batch workload's range: molecules whose orbitals fit one
    128-row tile (the CTA-pair tile is available and timed against the single-CTA tile), and
    the same mix with its last molecule of 130 orbitals (only the single-CTA tile exists).
    Each mix's tuned batch reproduces its single builds bit for bit."""
    s = 5
    mixes = {"small-nocc": [(30, 41), (52, 42), (75, 43), (100, 44)],
             "one-large-nocc": [(30, 41), (52, 42), (75, 43), (130, 45)]}
    chosen = {}
    for name, mols in mixes.items():
        ctxs, keep, Cs = [], [], []
        for atoms, seed in mols:
            mol = inputs.molecule(atoms, seed)
            B = inputs.df_tensor_device(mol)
            ctx = df.Context(mol.nao, mol.naux, atoms, s_max=s)
            ctx.setup(B)
            ctxs.append(ctx)
            keep.append(B)
            Cs.append(torch.from_numpy(inputs.orbitals(mol.nao, atoms, seed + 1)).cuda())
        single = [ctx.build_K(C, s)[0].clone() for ctx, C in zip(ctxs, Cs)]
        batch = df.Batch(ctxs)
        Ks = [torch.empty_like(k) for k in single]
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            chosen[name] = batch.autotune(Cs, s, Ks)
            batch.build_K(Cs, s, Ks)
        stream.synchronize()
        for k, k1 in zip(Ks, single):
            assert torch.equal(k, k1)
    print("autotuner choices (K-split cap, order, first-GEMM tile):", chosen)
    assert chosen["one-large-nocc"][2] == 0 and chosen["small-nocc"][2] in (0, 1)


def test_batch_side_streams_join_the_callers_stream(df, molecules):
    """Six molecules over the four side streams (two streams carry two molecules), with and
    without graphs: copies enqueued on the caller's stream right after a build see every
    molecule's finished K and J; a batch that names one context twice is refused."""
    s = 4
    mols = list(molecules)
    for atoms, seed in [(16, 21), (27, 22)]:
        mol = inputs.molecule(atoms, seed)
        C = inputs.orbitals(mol.nao, atoms, seed + 1)
        mols.append((inputs.df_tensor(mol), C, inputs.density(C)))
    ctxs, keep = [], []
    for B, C, D in mols:
        ctx = df.Context(B.shape[1], B.shape[0], C.shape[1], s_max=s)
        Bg = torch.from_numpy(B).cuda()
        ctx.setup(Bg)
        ctxs.append(ctx)
        keep.append(Bg)
    Cs = [torch.from_numpy(C).cuda() for _, C, _ in mols]
    Ds = [torch.from_numpy(D).cuda() for _, _, D in mols]
    single = [ctx.build_K(C, s)[0].clone() for ctx, C in zip(ctxs, Cs)]
    Js1 = [ctx.build_J(D)[0].clone() for ctx, D in zip(ctxs, Ds)]
    with pytest.raises(RuntimeError):
        df.Batch([ctxs[0], ctxs[1], ctxs[0]])
    batch = df.Batch(ctxs)
    stream = torch.cuda.Stream()
    for graphs in (True, False):
        batch.set_graphs(graphs)
        Ks = [torch.full_like(k, float("nan")) for k in single]
        Js = [torch.full_like(j, float("nan")) for j in Js1]
        with torch.cuda.stream(stream):
            for _ in range(2):
                batch.build_K(Cs, s, Ks, stream=stream)
                Kc = [k.clone() for k in Ks]
                batch.build_J(Ds, Js, stream=stream)
                Jc = [j.clone() for j in Js]
        stream.synchronize()
        for k, k1 in zip(Kc, single):
            assert torch.equal(k, k1)
        for j, j1 in zip(Jc, Js1):
            assert torch.equal(j, j1)
