"""The learned potential end to end (Sec. 4.1): training data from the
plain SW simulator (GPU Langevin at 500-3000 K), training of the BP network
by the hand-written double-backward kernels, and what it gains over the
method without it -- the SW two-body term alone and the untrained network."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    import paper_1912_04232_b300.learned as LP
    temps = np.linspace(500.0, 3000.0, 8)
    ds = LP.generate_sw_dataset(temps, n_snap=40, stride=20, equil=500, seed=1)
    LP.build_lists(ds)
    S = ds.r.shape[0]
    n_train = int(0.8 * S)
    tr = LP.Trainer(ds, batch=8, lr=3e-3, wF=1.0, seed=0)
    untrained = tr.evaluate(n_train, S)
    tr.train(0, n_train, epochs=60, seed=0, lr_end=1e-4)
    trained = tr.evaluate(n_train, S)
    two_body = LP.force_rmse_sw2body(ds, n_train, S)
    return dict(ds=ds, untrained=untrained, trained=trained, two_body=two_body, trainer=tr)


def test_dataset_is_physical(trained):
    ds = trained["ds"]
    e = (ds.E.cpu().numpy() / ds.n)
    # diamond SW cohesive energy -4.3366 eV/atom at 0 K; hotter = higher
    assert np.all(e > -4.34) and np.all(e < -3.0)
    hot = e[ds.T >= 2500].mean()
    cold = e[ds.T <= 900].mean()
    assert hot > cold + 0.2


def test_trained_network_beats_two_body_and_untrained(trained):
    fr = trained["trained"][1]
    print("force RMSE eV/A: trained %.4f untrained %.4f two-body %.4f; energy RMSE trained %.4f eV/atom"
          % (fr, trained["untrained"][1], trained["two_body"], trained["trained"][0]))
    assert fr * 5.0 <= trained["untrained"][1]
    assert fr * 5.0 <= trained["two_body"]


def test_deploy_at_64000_atoms(trained):
    # the trained network in NVE at N = 64,000 (20^3 diamond cells, 1000 K)
    # beside plain SW: both run, the learned forces stay close to SW
    import paper_1912_04232_b300.learned as LP
    tr = trained["trainer"]
    out = LP.deploy_compare(tr.params, tr.norm, n_side=20, T=1000.0, steps=100, warmup=10)
    print(out)
    assert out["N"] == 64000
    assert out["sw_particle_steps_per_s"] > 0 and out["learned_tc_particle_steps_per_s"] > 0
    assert out["force_rmse_vs_sw_start_eV_per_A"] < 3 * trained["trained"][1] + 0.05
    assert out["force_rmse_vs_sw_final_eV_per_A"] < 3 * trained["trained"][1] + 0.1
