"""What the trained face-value network gains over plain PPM (reading R14).

A small, deterministic version of the learned experiment: fine C96 x 4-level
runs (training seeds 11-14) coarsened 4x to C24 give the training samples;
the network is trained with the library's tensor-core gradient kernel; then
plain and learned C24 runs from an evaluation seed (1001) are compared
against the coarsened C96 truth after 240 substeps.  The tracers (pure
transport) are where the face values matter; delp and pt are dominated by the
coarse dynamics and must not get worse.  The learned face value is the plain
PPM value plus the network's correction, so a network that learned nothing
reproduces plain PPM."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_learned_gain_over_plain():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_04148_gb300 import learned
    res, w = learned.experiment(npx=24, r=4, nz=4, train_seeds=(11, 12, 13, 14), snapshots=8, every=6,
                                per_field=2000, nq=4, eval_seeds=(1001,), substeps=240, steps=800)
    # the network explains part of the correction the fine grid asks for
    assert res["sample_mse_network"] < res["sample_mse_plain"], (res["sample_mse_network"], res["sample_mse_plain"])
    ev = res["eval"][0]
    plain, learn = ev["plain"]["rel_rms_err"], ev["learned"]["rel_rms_err"]
    qp = np.mean([plain["q%d" % k] for k in range(4)])
    ql = np.mean([learn["q%d" % k] for k in range(4)])
    print("tracer rel. RMS error: plain %.5g learned %.5g (gain %.1f%%)" % (qp, ql, 100 * (1 - ql / qp)))
    print("wall s: plain %.3f learned %.3f" % (ev["plain"]["wall_s"], ev["learned"]["wall_s"]))
    assert ql < qp
    for f in ("delp", "pt"):
        assert learn[f] <= 1.02 * plain[f], (f, learn[f], plain[f])
