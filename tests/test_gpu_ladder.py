"""Adaptive N_seg ladder on the GPU: stages keep the same templates as selecting by the
oracle's statistic would, the injection survives to the last stage, and a run resumes
from its checkpoints with identical results."""
import numpy as np
import pytest

from paper_2510_19047_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ae45():
    return synth.two_year_two_channel(seed=77, n_inj=3, n_tranche=384, L=2048)


def ctx_for(D):
    from paper_2510_19047_b300.binding import TFS
    c = TFS(0, pn_order=D.pn_order, response=D.response, pixel="f32")
    c.load_tf_data(D.d, D.dt, D.dT, D.t0)
    c.set_noise_weights(D.w, D.mask)
    return c


def test_ladder_stages_and_resume(ae45, tmp_path):
    from paper_2510_19047_b300.ladder import run_ladder
    D = ae45
    bank = synth.two_year_bank(20_000, seed=31)
    bank[:, 12_345] = D.injections[:, 0]  # the loudest-by-construction template
    c = ctx_for(D)
    res = run_ladder(c, bank, stages=(128, 32, 8), keep=0.05, checkpoint_dir=str(tmp_path),
                     tag="t", seed=31)
    assert [r["n_seg"] for r in res] == [128, 32, 8]
    assert [len(r["index"]) for r in res] == [1000, 50, 2]
    assert 12_345 in res[-1]["index"]
    # stage 1 keeps exactly the top 5 % by (Upsilon desc, index asc)
    u, _, _ = c.eval_statistic(bank, 128)
    ref = np.lexsort((np.arange(u.size), -u))[:1000]
    assert np.array_equal(res[0]["index"], ref)
    # survivors of each stage are a subset of the previous stage's
    assert set(res[1]["index"]) <= set(res[0]["index"])
    assert set(res[2]["index"]) <= set(res[1]["index"])
    # resume: every stage is read back from the checkpoints
    res2 = run_ladder(c, bank, stages=(128, 32, 8), keep=0.05, checkpoint_dir=str(tmp_path),
                      tag="t", seed=31)
    assert all(r["resumed"] for r in res2)
    for a, b in zip(res, res2):
        assert np.array_equal(a["index"], b["index"]) and np.array_equal(a["stat"], b["stat"])
