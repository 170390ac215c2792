"""boruta_fit_batch: uneven jobs run together give, job by job, the oracle's
results (with the job's id keying its random streams) and the same results
as boruta_fit on the job alone."""
import numpy as np
import pytest

import oracle
from paper_2605_09950_gb300 import synth

pytestmark = pytest.mark.gpu


def _jobs():
    ws = synth.batch_jobs(n_jobs=5, n_trees=12, max_depth=6, max_iter=6, N_range=(200, 2000), p_range=(5, 40))
    ws.append(synth.snp_regression(N=700, p=25, n_add=4, n_pairs=2, n_trees=8, max_depth=6, max_iter=6))
    ws.append(synth.binary_small(N=500, p=12, n_inf=3, n_trees=10, max_depth=6, max_iter=6, importance=0))
    return ws


def test_batch_matches_oracle_and_single_fits():
    import torch

    import __graft_entry__
    from paper_2605_09950_gb300 import boruta

    __graft_entry__.build()
    ws = _jobs()
    jobs = []
    for w in ws:
        params = w.params()
        jobs.append(dict(X=torch.from_numpy(w.X).cuda(), y=torch.from_numpy(w.y).cuda(), N=w.N, **params))
    outs = boruta.boruta_fit_batch(jobs, job=3)
    for j, (w, got) in enumerate(zip(ws, outs)):
        params = w.params()
        want = oracle.BorutaProblem(w.X, w.y, **params, N=w.N, job=3 + j).run()
        assert got["iterations"] == want["iterations"], j
        np.testing.assert_array_equal(got["decision"], want["decision"], err_msg=f"job {j}")
        np.testing.assert_array_equal(got["hits"], want["hits"], err_msg=f"job {j}")
        if (w.task & 2) == 0 or (w.task & 1) == 1:  # exact sums: bit-exact history
            np.testing.assert_array_equal(got["imp_history"], want["imp_history"], err_msg=f"job {j}")
        nc = params.pop("n_classes")
        single = boruta.boruta_fit(jobs[j]["X"], jobs[j]["y"], N=w.N, n_classes=nc, job=3 + j, **params)
        np.testing.assert_array_equal(single["imp_history"], got["imp_history"])


def test_batch_reports_the_failing_job():
    import torch

    from paper_2605_09950_gb300 import boruta

    w = synth.binary_small(N=100, p=5, n_inf=1, n_trees=3, max_depth=3, max_iter=2)
    good = dict(X=torch.from_numpy(w.X).cuda(), y=torch.from_numpy(w.y).cuda(), N=w.N, **w.params())
    bad = dict(good, n_bins=1)
    with pytest.raises(boruta.BorutaError, match="job 1"):
        boruta.boruta_fit_batch([good, bad])


def test_stepwise_batch_matches_fit_batch():
    import torch

    import __graft_entry__
    from paper_2605_09950_gb300 import boruta

    __graft_entry__.build()
    ws = _jobs()[:4]
    jobs = [dict(X=torch.from_numpy(w.X).cuda(), y=torch.from_numpy(w.y).cuda(), N=w.N, **w.params()) for w in ws]
    want = boruta.boruta_fit_batch(jobs, job=7, precision=1)
    B = boruta.Batch(jobs, job=7, precision=1)
    steps, running = 0, len(jobs)
    while running:
        running = B.step()
        steps += 1
    assert steps == max(o["iterations"] for o in want)
    for j in range(len(jobs)):
        got = B.read(j)
        assert got["iterations"] == want[j]["iterations"]
        for key in ("decision", "hits", "imp_history", "shadow_max"):
            np.testing.assert_array_equal(got[key], want[j][key], err_msg=f"job {j} {key}")
    with pytest.raises(boruta.BorutaError, match="finished"):
        B.step()
    B.close()
    # free-running: two iterations at a time, jobs advancing independently
    R = boruta.Batch(jobs, job=7, precision=1)
    while R.run(2):
        pass
    for j in range(len(jobs)):
        got = R.read(j)
        for key in ("decision", "hits", "imp_history", "shadow_max"):
            np.testing.assert_array_equal(got[key], want[j][key], err_msg=f"job {j} {key}")
    R.close()


def test_fit_seeds_matches_oracle_runs_and_median_selection():
    """boruta_fit_seeds: the seeds run as jobs of one batch; every run equals
    the oracle's run with that seed (and job id), and the median selection
    and the final ranking of each run equal the oracle's."""
    import torch

    import __graft_entry__
    from paper_2605_09950_gb300 import boruta

    __graft_entry__.build()
    w = synth.paper_regression("direct", N=600, n_trees=12, max_depth=6, max_iter=8, importance=synth.TREEIMP,
                               mtry=0)
    seeds = [3, 17, 29, 41, 57]
    params = w.params()
    params.pop("seed")
    nc = params.pop("n_classes")
    runs, med, ms, sel = boruta.boruta_fit_seeds(torch.from_numpy(w.X).cuda(), torch.from_numpy(w.y).cuda(),
                                                 seeds=seeds, N=w.N, n_classes=nc, job=2, **params)
    want = []
    for j, sd in enumerate(seeds):
        o = oracle.BorutaProblem(w.X, w.y, **{**w.params(), "seed": sd}, N=w.N, job=2 + j).run()
        g = runs[j]
        assert g["iterations"] == o["iterations"]
        for key in ("decision", "hits", "imp_history", "shadow_max"):
            np.testing.assert_array_equal(g[key], o[key], err_msg=f"seed {sd} {key}")
        np.testing.assert_array_equal(boruta.boruta_rank(g["decision"], g["imp_history"], g["iterations"]),
                                      oracle.rank(o["decision"], o["imp_history"], o["iterations"]))
        want.append(o)
    om, oms, osel = oracle.select_median(want)
    np.testing.assert_array_equal(med, om)
    assert ms == oms
    np.testing.assert_array_equal(sel, osel)
    assert sel[w.informative].sum() >= 5  # the strong target variables stand out already at this size
