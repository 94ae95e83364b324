"""pa_energies (device evaluation of host configurations) against the oracle's
energy, and the verify command line on a G-set file."""
import json
import subprocess
import sys

import numpy as np
import pytest

import oracle
from gpu_helpers import require_gpu
from paper_2510_21105_gb300 import binding as B
from paper_2510_21105_gb300 import hexconfig
from paper_2510_21105_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("g", [wl.gnp(301, 0.05, seed=11), wl.torus(13, seed=12), wl.delaunay(777, seed=13),
                               wl.gnm(7000, 41459, seed=0)], ids=["gnp", "torus", "delaunay", "g63like"])
def test_energies_match_oracle(g):
    require_gpu()
    rng = np.random.default_rng(5)
    x = np.where(rng.random((9, g.n)) < 0.5, 1, -1).astype(np.int8)
    x[0] = 1                               # all equal: E = W, cut 0
    with B.Annealer.from_graph(g) as ann:
        E, cuts = ann.energies(x)
        W = ann.stats()["total_weight"]
        E0, _ = ann.energies(x[:0])
    ref = np.array([oracle.energy(g.rp, g.col, g.w, xi) for xi in x])
    assert np.array_equal(E, ref)
    assert np.array_equal(cuts, (W - ref) // 2)
    assert cuts[0] == 0 and len(E0) == 0


def test_energies_rejects_bad_spins():
    require_gpu()
    g = wl.gnp(40, 0.2, seed=1)
    with B.Annealer.from_graph(g) as ann:
        with pytest.raises(RuntimeError):
            ann.energies(np.zeros((1, g.n), np.int8))


def test_verify_cli_on_annealed_configuration(tmp_path):
    require_gpu()
    g = wl.gnm(500, 3000, seed=21)
    gp = tmp_path / "g.txt"
    wl.write_gset(g, str(gp))
    hp = tmp_path / "best.hex"
    run = subprocess.run([sys.executable, "-m", "paper_2510_21105_gb300.cli", "--graph", str(gp),
                          "--replicas", "256", "--sweeps", "2", "--beta", "0.1", "2.0", "20",
                          "--nlm-period", "5", "--save-hex", str(hp)], capture_output=True, text=True,
                         check=True)
    best = json.loads(run.stdout.strip().splitlines()[-1])["best_cut"]
    x = hexconfig.decode(hp.read_text(), g.n)
    assert (oracle.total_weight(g.rp, g.col, g.w) - oracle.energy(g.rp, g.col, g.w, x)) // 2 == best
    ok = subprocess.run([sys.executable, "-m", "paper_2510_21105_gb300.cli", "verify", "--graph", str(gp),
                         "--hex-file", str(hp), "--expect-cut", str(best)], capture_output=True, text=True)
    assert ok.returncode == 0 and json.loads(ok.stdout)["cut"] == best
    bad = subprocess.run([sys.executable, "-m", "paper_2510_21105_gb300.cli", "verify", "--graph", str(gp),
                          "--hex-file", str(hp), "--expect-cut", str(best + 1)], capture_output=True, text=True)
    assert bad.returncode == 1


def _cli(*args):
    run = subprocess.run([sys.executable, "-m", "paper_2510_21105_gb300.cli", *map(str, args)],
                         capture_output=True, text=True, check=True)
    return json.loads(run.stdout.strip().splitlines()[-1])


def test_cli_checkpoint_resume_and_curve(tmp_path):
    """Long-run mode: a run stopped after 10 of 20 steps and resumed from its
    checkpoint reports the same best cut and the same cut-vs-step curve as
    the uninterrupted run; the curve is monotone and ends at the best cut."""
    require_gpu()
    g = wl.gnm(600, 4000, seed=31)
    gp = tmp_path / "g.txt"
    wl.write_gset(g, str(gp))
    common = ["--graph", gp, "--replicas", 512, "--sweeps", 2, "--beta", 0.1, 2.5, 20, "--nlm-period", 4,
              "--variant", 2]
    full = _cli(*common, "--curve", tmp_path / "full.csv")
    ck = tmp_path / "ck.bin"
    _cli(*common, "--steps", 10, "--checkpoint", ck, "--checkpoint-every", 4)
    res = _cli(*common, "--resume", ck, "--curve", tmp_path / "res.csv")
    assert res["best_cut"] == full["best_cut"] and res["best_step"] == full["best_step"]
    c_full = np.loadtxt(tmp_path / "full.csv", delimiter=",", skiprows=1)
    c_res = np.loadtxt(tmp_path / "res.csv", delimiter=",", skiprows=1)
    assert c_full.shape == c_res.shape == (20, 4)
    assert np.array_equal(c_full[:, [0, 1, 3]], c_res[:, [0, 1, 3]])
    assert np.all(np.diff(c_full[:, 3]) >= 0) and c_full[-1, 3] == full["best_cut"]
    assert np.all(np.diff(c_full[:, 2]) >= 0)


def test_cli_adaptive_modes_equal_the_api(tmp_path):
    """The CLI's adaptive-control options (ESS-adaptive steps, acceptance-rate
    steps, stagnation reheating) run the same anneal as the Python API with
    the same options: same steps, best cut and where it was found."""
    require_gpu()
    g = wl.gnm(500, 3000, seed=41)
    gp = tmp_path / "g.txt"
    wl.write_gset(g, str(gp))
    common = ["--graph", gp, "--replicas", 256, "--sweeps", 2, "--beta", 0.1, 2.0, 60, "--variant", 2,
              "--nlm-period", 0]
    cases = [
        (["--adaptive", 1, "--rho", 0.6, "--adapt-J", 6, "--dbeta-max", 0.2],
         dict(adaptive=1, rho=0.6, adapt_J=6, adapt_dbeta_max=0.2, beta_max=2.0, acc_lo=0.05, acc_hi=0.25)),
        (["--adaptive", 2, "--adapt-J", 5, "--dbeta-max", 0.3, "--acc-lo", 0.1, "--acc-hi", 0.3],
         dict(adaptive=2, rho=0.5, adapt_J=5, adapt_dbeta_max=0.3, beta_max=2.0, acc_lo=0.1, acc_hi=0.3)),
        (["--reheat-after", 3, "--reheat-back", 5], dict(reheat_after=3, reheat_back=5)),
    ]
    betas = wl.linear_betas(0.1, 2.0, 60)
    for args, kw in cases:
        out = _cli(*common, *args)
        with B.Annealer.from_graph(g) as a:
            a.anneal(None if kw.get("adaptive") else betas, 256, 2, 0, K=60, nlm_period=0, **kw)
            st = a.stats()
            E, step, sweep, slot = a.best_record()
        assert out["steps"] == st["steps_run"]
        assert out["best_cut"] == (st["total_weight"] - E) // 2 and out["best_step"] == step, args
