"""What the trained proposal network (paper_2607_16897_gb300/proposal_weights.npy,
trained on the GPU by ``python -m paper_2607_16897_gb300.proposal`` on seeds
10000-11023) gains over the plain method on held-out sequences (seeds 5000+),
in a paired comparison from the same constant-velocity starts: its starts are
closer to the converged states, the full LM after it reaches the plain form's
final poses, and it does not add linearisation passes.  The statistics are
printed (pytest -s)."""
import json

import pytest

pytestmark = pytest.mark.gpu


def test_trained_proposal_gain_on_held_out_sequences():
    from paper_2607_16897_gb300 import proposal as prop
    st = prop.evaluate(prop.load_weights(), seeds=range(prop.TEST_SEED0, prop.TEST_SEED0 + 48),
                       frames=16)
    print(json.dumps(st))
    assert st["frames"] == 48 * 14
    assert st["proposal_start_err"] < st["cv_start_err"]
    assert st["agree_1e5"] == 1.0
    assert st["passes_proposal"] <= st["passes_plain"] + 0.05
