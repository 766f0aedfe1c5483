"""Host-side helpers of bench.py, checked without a GPU: the headline guess is described and
its launches counted; the committed ncu traffic is reported only while the measured
kernel's sources are unchanged; the pair count and the replica grid rule follow their
definitions; the clock sampler's parser reports the median clock and the throttle reasons
that were active; the host-core harness that times the oracle reproduces the serial oracle."""
import json
import os
import shutil

import numpy as np

import bench

REPO = bench.ROOT


def test_guess_tables_cover_the_headline():
    for k in (bench.HEADLINE_GUESS, "learned+adaptive", "learned+extrapolated"):
        assert k in bench.GUESS_TEXT and k in bench.GUESS_LAUNCHES
    # the adaptive predictor is the hold plus one reduction kernel
    assert bench.GUESS_LAUNCHES["learned+adaptive"] == bench.GUESS_LAUNCHES["learned+previous"] + 1


def test_launch_count_grows_seven_per_iteration():
    a = bench.launches_per_step(4, 96000, 0.0, 6)
    assert bench.launches_per_step(5, 96000, 0.0, 6) - a == 7
    assert bench.launches_per_step(4, 96001, 0.0, 6) - a == 1      # padding kernel for a ragged tail
    assert bench.launches_per_step(4, 96000, 1.0, 6) - a == 14     # a list rebuild every step


def _copy_profile_tree(dst):
    src = os.path.join(REPO, "profiles", "real_matvec_water96k.json")
    with open(src) as fh:
        d = json.load(fh)
    os.makedirs(os.path.join(dst, "profiles"))
    shutil.copy(src, os.path.join(dst, "profiles"))
    for f in d["sources"]:
        os.makedirs(os.path.dirname(os.path.join(dst, f)), exist_ok=True)
        shutil.copy(os.path.join(REPO, f), os.path.join(dst, f))
    return d


def test_captured_traffic_tracks_the_kernel_sources(tmp_path, monkeypatch):
    d = _copy_profile_tree(str(tmp_path))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the copy carries the committed sources: the figure is valid exactly when the hash of
    # the committed sources equals the one stored with the capture
    with open(os.path.join(str(tmp_path), "profiles", "real_matvec_water96k.json")) as fh:
        stored = json.load(fh)
    got = bench.captured_traffic()
    assert got in (None, d["dram_bytes_per_launch"])
    stored["source_sha256_16"] = "0" * 16                              # a capture of other sources
    with open(os.path.join(str(tmp_path), "profiles", "real_matvec_water96k.json"), "w") as fh:
        json.dump(stored, fh)
    assert bench.captured_traffic() is None
    if got is not None:                                                # one changed byte voids it
        _copy_profile_tree(str(tmp_path / "b"))
        monkeypatch.setattr(bench, "ROOT", str(tmp_path / "b"))
        assert bench.captured_traffic() == d["dram_bytes_per_launch"]
        with open(os.path.join(str(tmp_path / "b"), d["sources"][0]), "ab") as fh:
            fh.write(b"\n")
        assert bench.captured_traffic() is None


def test_pairs_within_against_brute_force():
    rng = np.random.default_rng(5)
    box, rc = 9.0, 3.1
    xyz = rng.uniform(-box, 2 * box, size=(200, 3))                    # images outside the box too
    d = xyz[:, None, :] - xyz[None, :, :]
    d -= box * np.round(d / box)
    r = np.sqrt((d ** 2).sum(-1))
    want = int(((r < rc) & np.triu(np.ones_like(r, dtype=bool), 1)).sum())
    assert bench.pairs_within(xyz, box, rc) == want


def test_smooth7_rule():
    good = [k for k in range(2, 130) if bench._smooth7(k)]
    assert good[:12] == [2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15]
    assert not any(bench._smooth7(k) for k in (11, 13, 22, 26, 121))
    assert all(bench._smooth7(k) for k in (100, 224, 64, 126))


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_parser_reports_median_and_reasons(tmp_path):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    c.fh = open(c.path, "w")
    c.fh.write("2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active\n"
               "2062, 2070, 1190.5, Not Active, Not Active, Not Active, Active\n"
               "1995, 2070, 1201.0, Not Active, Active, Not Active, Active\n"
               "[N/A], 2070, 0, Not Active, Not Active, Not Active, Not Active\n"
               "garbage\n")
    c.fh.flush()
    c.proc = _DoneProc()
    got = c.stop()
    assert got["sm_mhz"] == 2062.0 and got["sm_max_mhz"] == 2070.0 and got["samples"] == 3
    assert got["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert not os.path.exists(c.path)


def test_trajectory_is_seeded():
    from paper_2011_01207_gb300 import synth
    s = synth.water_box(27, 9.3, 11)
    a, b = bench.trajectory(s, 4), bench.trajectory(s, 4)
    assert a.shape == (4, s.n, 3) and np.array_equal(a, b)
    assert np.array_equal(a[0], s.xyz) and not np.array_equal(a[1], a[0])


def test_clock_sampler_without_nvidia_smi_leaves_no_file():
    c = bench.Clocks(0)
    c.proc = None
    assert os.path.exists(c.path)
    got = c.stop()
    assert got["sm_mhz"] is None and not os.path.exists(c.path)


def test_host_oracle_harness_equals_serial_oracle():
    """The host-core harness that times the oracle only splits the oracle's own pair sums and
    smooth-PME passes over worker processes: field, PCG iterates, energy and forces equal the
    serial oracle's to rounding (the parts are summed in another order), and the module
    references it swaps are restored afterwards."""
    import oracle.model as om
    from oracle import Oracle, Params
    from paper_2011_01207_gb300 import synth
    s = synth.water_box(64, 12.5, 4242, dmin_inter=1.7)
    p = Params(beta=0.5446, grid=(16, 16, 16), cutoff=6.0)
    o = Oracle(s, p)
    E = o.permanent_field()
    mu, info = o.pcg(E, tol=1e-6)
    e_ref, F_ref = o.energy(mu, E), o.forces(mu)
    saved = (om.pairs, om.realspace, om.spme)
    h = bench.HostOracle(3)
    h.start(s.n)
    try:
        _, iters, _, (E2, mu2, e2, F2) = h.step(s, p, 1e-6, outputs=True)
        E3, resid, e3, F3, V3 = h.at_dipoles(s, p, mu)
    finally:
        h.stop()
    np.testing.assert_allclose(E3, E, rtol=1e-11, atol=1e-13)
    assert abs(resid - o.residual_eps(E - o.apply_A(mu))) < 1e-12
    assert abs(e3 - e_ref) < 1e-12 * abs(e_ref)
    np.testing.assert_allclose(F3, F_ref, rtol=1e-10, atol=1e-11)
    V = o.virial(mu)
    np.testing.assert_allclose(V3, V, rtol=1e-9, atol=1e-10 * np.abs(V).max())
    assert (om.pairs, om.realspace, om.spme) == saved
    assert iters == info["iters"]
    np.testing.assert_allclose(E2, E, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(mu2, mu, rtol=1e-9, atol=1e-12)
    assert abs(e2 - e_ref) < 1e-10 * abs(e_ref)
    np.testing.assert_allclose(F2, F_ref, rtol=1e-9, atol=1e-10)
