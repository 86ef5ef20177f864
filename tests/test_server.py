"""Serving loop: admission by footprint, concurrency and result equality.

The scheduler tests run on the CPU in the server's dry-run mode (workers
hold their slot for a time that grows with the request, without GPU work).
The GPU test checks that requests run concurrently and that every result is
bit-identical to the same request solved alone."""
import time

import numpy as np
import pytest

from paper_2208_01348_gb300 import inputs as I


@pytest.fixture(scope="module")
def dd():
    from paper_2208_01348_gb300 import build
    build.build()
    from paper_2208_01348_gb300 import eelsdda
    return eelsdda


def _request(n, n_energy, n_beam):
    occ = I.sphere_occupancy(n, n * 1.25)
    e = np.linspace(1.5, 3.5, n_energy)
    beams = np.stack([np.full(n_beam, n * 0.625 + 3.0), np.linspace(-1, 1, n_beam)], axis=1)
    return occ, 1.25, e, I.drude(e)[:, None], np.full(n_energy, 2.1 + 0j), beams


def test_dryrun_admission_respects_budget_and_backfills(dd):
    o = dd.eels_default_opts()
    # 64 x 8 points: the dry run holds each big request's slot for ~10 ms, far
    # longer than submitting the next requests takes
    occ_big, d, e, ep, eh, b = _request(24, 64, 8)
    fp_big = dd.eels_query_footprint(occ_big, d, o, 1)     # smallest batch of the big request
    budget = int(fp_big * 1.5)       # room for one big request at a time, plus small ones
    srv = dd.eels_server_create(hbm_budget=budget, max_concurrent=2, flags=dd.EELS_SERVER_DRYRUN)
    try:
        jobs = [dd.eels_server_submit(srv, occ_big, d, o, e, ep, eh, b) for _ in range(2)]
        occ_s, d_s, e_s, ep_s, eh_s, b_s = _request(8, 2, 1)
        small = dd.eels_server_submit(srv, occ_s, d_s, o, e_s, ep_s, eh_s, b_s)
        infos = {}
        peak = 0
        while len(infos) < 3:
            st = dd.eels_server_stats(srv)
            assert st["in_use"] <= budget
            peak = max(peak, st["in_use"])
            for j in jobs + [small]:
                i = dd.eels_server_poll(srv, j)
                if i["state"] == dd.EELS_JOB_DONE:
                    infos[j] = i
            time.sleep(0.0005)
        big0, big1, sm = infos[jobs[0]], infos[jobs[1]], infos[small]
        # the second big request waits for the first (budget), the small one passes it
        assert big1["t_start"] >= big0["t_end"] - 1e-6
        assert sm["t_start"] < big1["t_start"]
        assert dd.eels_server_stats(srv)["running_max"] == 2
    finally:
        dd.eels_server_destroy(srv)


def test_dryrun_rejects_requests_larger_than_budget(dd):
    o = dd.eels_default_opts()
    occ, d, e, ep, eh, b = _request(24, 4, 2)
    fp1 = dd.eels_query_footprint(occ, d, o, 1)
    srv = dd.eels_server_create(hbm_budget=fp1 // 2, max_concurrent=1, flags=dd.EELS_SERVER_DRYRUN)
    try:
        with pytest.raises(dd.EelsError) as ex:
            dd.eels_server_submit(srv, occ, d, o, e, ep, eh, b)
        assert ex.value.code == dd.EELS_E_OOM
    finally:
        dd.eels_server_destroy(srv)


def test_dryrun_fifo_when_everything_fits(dd):
    o = dd.eels_default_opts()
    occ, d, e, ep, eh, b = _request(10, 4, 2)
    srv = dd.eels_server_create(hbm_budget=1 << 40, max_concurrent=1, flags=dd.EELS_SERVER_DRYRUN)
    try:
        ids = [dd.eels_server_submit(srv, occ, d, o, e, ep, eh, b) for _ in range(5)]
        starts = [dd.eels_server_wait(srv, j, len(e), len(b))[2]["t_start"] for j in ids]
        assert starts == sorted(starts)
    finally:
        dd.eels_server_destroy(srv)


@pytest.mark.gpu
def test_requests_overlap_and_match_solo_results(dd):
    reqs = [_request(12, 6, 3), _request(16, 4, 2), _request(10, 8, 1), _request(14, 3, 4)]
    o = dd.eels_default_opts(ekin_keV=100.0, eps_it=1e-8)
    solo = []
    ctx = dd.eels_create(0)
    try:
        for occ, d, e, ep, eh, b in reqs:
            dd.eels_set_grid(ctx, occ, d)
            solo.append(dd.eels_solve(ctx, o, e, ep, eh, b))
    finally:
        dd.eels_destroy(ctx)
    srv = dd.eels_server_create(device=0, max_concurrent=3)
    try:
        ids = [dd.eels_server_submit(srv, occ, d, o, e, ep, eh, b) for occ, d, e, ep, eh, b in reqs]
        for j, (occ, d, e, ep, eh, b), ref in zip(ids, reqs, solo):
            code, out, info = dd.eels_server_wait(srv, j, len(e), len(b))
            assert code == dd.EELS_OK and info["state"] == dd.EELS_JOB_DONE
            assert np.array_equal(out["eels"], ref.p_eels)
            assert np.array_equal(out["cl"], ref.p_cl)
            assert np.array_equal(out["ext"], ref.p_ext)
        assert dd.eels_server_stats(srv)["running_max"] >= 2
    finally:
        dd.eels_server_destroy(srv)
