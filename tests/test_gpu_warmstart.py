"""What the trained network gains over plain PLS-TV: the learned warm-start experiment end to
end at 32^3 (48 training and 6 held-out phantoms, 60 epochs; about a minute on one GB300).
Zero-start FISTA-TV is the reference and the yardstick: both runs must reach the 1e-3 relative data
residual, and the warm start must get there in fewer iterations and less GPU time (its network
and amplitude fit included)."""
import pytest

pytestmark = pytest.mark.gpu


def test_learned_warm_start_beats_zero_start():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1304_2017_gb300 import warmstart
    s = warmstart.run(n_train=48, n_test=6, epochs=60, target_iters=200, max_iters=400, n=32)
    print({k: v for k, v in s.items() if k != "per_phantom"})
    assert s["reached"].startswith("6 of 6"), s["reached"]
    assert s["train_loss_first_last"][1] < 0.1 * s["train_loss_first_last"][0]
    assert s["mean_warm_iters"] <= 0.95 * s["mean_zero_iters"], (s["mean_warm_iters"], s["mean_zero_iters"])
    assert s["mean_warm_gpu_s"] < s["mean_zero_gpu_s"], (s["mean_warm_gpu_s"], s["mean_zero_gpu_s"])
