"""bench.py's host-side helpers, no GPU: the FIFO queue the serving baselines
replay, the per-key reuse of measured service times, the whole-job
throughput, and the compact summary the bench line carries."""
import json
import sys
import types

import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_fifo_latencies_replay_one_solver_in_arrival_order():
    # arrivals 0, 1, 1.5 with service 2, 1, 1: completions 2, 3, 4
    assert bench.fifo_latencies([0.0, 1.0, 1.5], [2.0, 1.0, 1.0]) == [2.0, 2.0, 2.5]
    # an idle solver starts at the arrival
    assert bench.fifo_latencies([0.0, 10.0], [1.0, 1.0]) == [1.0, 1.0]


class _FakeCapi:
    """Records set-ups; a solve 'takes' no time, sequential stepping returns
    the problem's nx as its seconds (so reuse is visible)."""
    PREC_FP64 = 0

    class MgritOpts:
        @staticmethod
        def from_buffer_copy(o):
            return type("O", (), {"precision": None})()

    def __init__(self):
        self.setups = 0

    def mgrit_setup(self, prob, o, stream=None):
        self.setups += 1
        return prob

    def mgrit_solve(self, h, u0, out, allow_not_converged=False):
        return None, 0

    def mgrit_sequential(self, h, u0, fin):
        return float(h.nx)

    def mgrit_destroy(self, h):
        pass


def test_service_times_are_measured_once_per_key(monkeypatch):
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    monkeypatch.setattr(torch, "empty", lambda *a, **k: None)
    capi = _FakeCapi()
    reqs = [(types.SimpleNamespace(nx=nx), None, None) for nx in (256, 512, 256, 256, 1024)]
    keys = [("ERK", 1, r[0].nx) for r in reqs]
    cache = {}
    fp64, seq = bench.alone_service_times(capi, reqs, None, keys, cache)
    assert capi.setups == 3 and len(fp64) == len(seq) == 5
    assert seq == [256.0, 512.0, 256.0, 256.0, 1024.0]
    assert fp64[2] == fp64[0] and fp64[3] == fp64[0]
    # a later rate with the same keys measures nothing new
    bench.alone_service_times(capi, reqs[:2], None, keys[:2], cache)
    assert capi.setups == 3
    # without keys every request is measured
    bench.alone_service_times(capi, reqs, None)
    assert capi.setups == 8


def test_whole_job_throughput_counts_all_replicas():
    # 2 replicas x 10 steps x 1e6 DOF over the slowest rank's 500 ms
    assert bench.replicas_value(2, 1e6, 10, 500.0) == pytest.approx(4e7)
    assert bench.replica_max(123.0, 1) == 123.0


def test_compact_summary_is_small_and_carries_the_headline_figures():
    extra = {
        "gpu_sequential_fp64": {"dof_per_s": 1.9e9}, "speedup_vs_gpu_sequential": 6.4,
        "fp64_vcycle_L4_m8": {"dof_per_s": 4.4e9}, "mixed_df_vcycle_L4_m8": {"dof_per_s": 2.3e10},
        "batch_uneven": {"dof_per_s": 4.0e9, "plain_fp64_alone_dof_per_s": 3.0e9,
                         "plain_fp64_alone_with_setup_dof_per_s": 1.4e9, "gpu_sequential_dof_per_s": 2.8e8,
                         "latency_ms": {"p50": 7500.0, "p99": 10000.0}, "converged": 4096},
        "batch_subset_vs_oracle": {"solves": 24, "err_vs_oracle": {"max": 6e-10},
                                   "iterations_minus_oracle": [0, 2], "gpu_batch_s": 10.05,
                                   "extrapolated_oracle_batch_s": {"subset_rate": 3175.2,
                                                                   "headline_sample_rate": 1682.4}},
        "sdirk3_u5_8192": {"mixed": {"ms": 24.9}, "fp64": {"ms": 39.6}, "gpu_sequential_fp64": {"ms": 873.0}},
    }
    out = bench.compact_summary(extra)
    assert out["speedup_vs_gpu_sequential"] == 6.4
    assert out["batch_4096"]["plain_fp64_alone"] == 3.0e9
    assert out["batch_subset_vs_oracle"]["oracle_batch_s_extrapolated"] == [3175, 1682]
    assert out["sdirk3_u5_8192_ms"]["mixed"] == 24.9
    assert len(json.dumps(out)) < 1500


def test_fourier_fcf_work_counts_every_butterfly():
    """bench.fourier_fcf_work (the roofline's FP64 work of the level-1 FCF's
    Fourier-space pass) against an enumeration of the passes' butterflies,
    for odd and even log2(nx/2)."""
    for nx in (8, 16, 256, 512, 4096, 8192):
        h = nx // 2
        ops = flops = 0
        spans = []
        q = h // 4
        while q >= 1:
            spans.append(q)
            q //= 4
        for _direction in range(2):
            for q in spans:
                for b in range(h // 4):
                    pos = b % q
                    ops += 16 + (12 if pos else 0)
                    flops += 16 + (18 if pos else 0)
            if (h.bit_length() - 1) % 2:
                ops += 4 * (h // 2)
                flops += 4 * (h // 2)
        for _k in range(h // 2 + 1):
            ops += 32
            flops += 40
        ops += 2 * nx
        flops += nx
        assert bench.fourier_fcf_work(nx) == (ops, flops), nx
