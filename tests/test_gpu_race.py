"""The learned-vs-plain race tool end to end on small instances (GPU): trace
collection, on-device training, Lanczos E0 and both arms on a Kitaev-chain
and a periodic Bose-Hubbard target.  Each arm's energy error may only fall
(every iteration appends a zero-angle gate to the previous optimum and BFGS
accepts only descent steps), and the learned arm spends fewer exact pool
gradients than the full screen."""
import pytest

from paper_2606_05297_gb300 import race

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("target,L", [("kitaev", 4), ("bh", 5)])
def test_race_runs_both_arms(target, L):
    out = race.main(["--target", target, "--L", str(L), "--d", "4", "--small-traces", "--trace-ops", "3",
                     "--train-steps", "5", "--max-ops", "6", "--hessian-recycling"])
    assert out["training"]["lists"] > 0 and out["training"]["loss_last"] is not None
    for arm in ("plain", "learned"):
        a = out[arm]
        assert 1 <= a["iterations"] <= 6
        dE = [h["dE"] for h in a["history"]]
        assert all(b <= e + 1e-9 * max(1.0, abs(out["target"]["E0"])) for e, b in zip(dE, dE[1:])), dE
        assert all(h["t"] > 0 for h in a["history"])
    assert out["learned"]["exact_gradients"] < out["plain"]["exact_gradients"]
    assert out["learned"]["full_screens"] >= 1
