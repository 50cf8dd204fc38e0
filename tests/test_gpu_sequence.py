"""The adaptive rule along the SCF-like sequence (GPU builds, oracle rule)."""
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


def test_adaptive_sequence_follows_table1_and_converges(df):
    from paper_2601_08077_gb300 import sequence
    mol, B, C, D = inputs.make_inputs(inputs.SMALL)
    ctx = df.Context(mol.nao, mol.naux, C.shape[1])
    Bg = torch.from_numpy(B).cuda()
    ctx.setup(Bg)
    orbs = sequence.orbital_sequence(C, 15, inputs.SMALL.seed)
    recs = sequence.run(ctx, orbs)
    levels = [r["level"] for r in recs]
    E = [r["E"] for r in recs]
    assert levels == O.level_schedule(E)[:len(levels)]
    assert all(a >= b for a, b in zip(levels, levels[1:]))
    assert levels[0] == 4 and levels[-1] <= 1
    # the early, low-precision iterations are far from FP64; the late ones agree closely
    assert recs[0]["max_dK_rel"] > 1e-9
    assert recs[-1]["dE_vs_fp64"] < 1e-9
    # every iteration runs its level's count in every block and meets that count's accuracy
    for r in recs:
        s = r["slices"][0]
        assert r["slices"] == [s] * r["nblk"] and s == O.slices_for_level(r["level"])
        if s:
            assert r["max_dK_rel"] < {3: 1e-5, 4: 1e-7, 5: 1e-10, 6: 1e-12}.get(s, 1e-13)
        assert r["fallback"] == (s == 0) and r["recomputed"] == 0
