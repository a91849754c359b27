"""Host-side arithmetic of the benchmark (no GPU): the algorithmic bytes per node update that
the roofline divides by, the committed DRAM-traffic figure and the source hash that guards it,
and the closed forms the benchmark reports errors against."""
import os
import sys

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")


def test_step_bytes_per_node_counts_each_stream_once():
    # FP32 difference form: weights of the K - 1 members other than the centre, 8 directions,
    # plus K - 1 int32 indices and 9 populations in and out
    assert bench.step_bytes_per_node(30, 4) == 8 * 29 * 4 + 29 * 4 + 18 * 4 == 1116
    # FP64 literal sum: all K members
    assert bench.step_bytes_per_node(30, 8) == 8 * 30 * 8 + 29 * 4 + 18 * 8 == 2180
    # nearest-node rule: K indices per direction
    assert bench.step_bytes_per_node(30, 4, nearest=True) == 8 * 29 * 4 + 8 * 30 * 4 + 72


def test_roofline_bytes_follow_the_scope_table_count():
    # shared stencil, K entries per direction and K indices: 36 K + 72 (FP32), 68 K + 144 (FP64)
    assert bench.survey_bytes_per_node(30, 4) == 36 * 30 + 72 == 1152
    assert bench.survey_bytes_per_node(30, 8) == 68 * 30 + 144 == 2184
    # the FP32 kernel's own count is 36 bytes less (no centre weight, no centre index)
    assert bench.survey_bytes_per_node(30, 4) - bench.step_bytes_per_node(30, 4) == 36


def test_adjoint_and_shan_chen_bytes_per_node():
    K = 24
    # reverse step: the forward's weights and indices once, s_next and lam_next in, lam_prev out
    assert bench.adjoint_bytes_per_node(K) == 8 * 23 * 4 + 23 * 4 + 3 * 36 == 936
    # two passes each reading the weights and indices; states, psi and the streamed states
    per_pass = 8 * 23 * 4 + 23 * 4
    assert bench.sc_bytes_per_node(K) == 2 * per_pass + 76 + 76


def test_committed_traffic_belongs_to_the_current_step_kernel():
    """The DRAM bytes per launch in the committed summary are used only while the step
    kernel's source hash equals the one recorded with them; when it does, the figure is that
    of one full-size launch and lies near the algorithmic bytes (a gather kernel that re-read
    its inputs would be far above)."""
    traffic = bench._ncu_traffic("f32")
    text = open(os.path.join(ROOT, "profiles", "step_f32_tgv_large.txt")).read()
    recorded = [ln.split(":", 1)[1].strip() for ln in text.splitlines() if ln.startswith("kernel_source_hash:")]
    assert len(recorded) == 1
    if recorded[0] != bench._step_source_hash():
        assert traffic is None
        pytest.skip("step kernel changed since the committed capture: traffic reported as null")
    n = 2048 * 2048
    algorithmic = bench.step_bytes_per_node(30, 4) * n
    assert 0.85 * algorithmic <= traffic <= 1.15 * algorithmic


def test_source_hash_ignores_comments_only():
    h = bench._step_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    assert bench._step_source_hash() == h  # deterministic


def test_annulus_profile_matches_the_oracle_closed_form():
    r1, r2, g, nu = 0.5 / 0.01, 1.0 / 0.01, 1e-6, bench.lattice_nu(0.7)
    r = np.linspace(r1, r2, 11)
    np.testing.assert_allclose(bench.annulus_profile(r, g, nu, r1, r2),
                               oracle.annulus_velocity(r, g, nu, r1, r2), rtol=1e-14, atol=0)
    assert abs(bench.annulus_profile(r1, g, nu, r1, r2)) < 1e-12
    assert abs(bench.annulus_profile(r2, g, nu, r1, r2)) < 1e-12


def test_lattice_viscosity_reading():
    assert bench.lattice_nu(0.8) == pytest.approx(0.1)
    assert bench.lattice_nu(0.8) == pytest.approx(oracle.lattice_viscosity(0.8))


def test_reference_line_names_the_sample_it_times(capsys):
    """The reference arm times the oracle on the bounded sample cloud, so its config names that
    cloud (128^2 nodes of the same recipe) and records which workload it samples."""
    import json
    import types

    cfg = bench._sample_config("tgv_large")
    c = bench.CPU_SAMPLE
    assert cfg["workload"] == f"tgv_{c['n_side']}sq_k{c['K']}_d{c['deg']}" == "tgv_128sq_k30_d4"
    assert cfg["nodes"] == 128 * 128
    assert cfg["sample_of"] == bench._config("tgv_large", 1)["workload"] == "tgv_2048sq_k30_d4"
    args = types.SimpleNamespace(steps=1, warmup=0, gpus=1, workload="tgv_large", ratio=1.0,
                                 stencil="own")
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["config"]["workload"] == "tgv_128sq_k30_d4" and line["config"]["nodes"] == 16384
    assert line["value"] == line["cpu_baseline"]["value"] == line["e2e"]["value"] > 0
