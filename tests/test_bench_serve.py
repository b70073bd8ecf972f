"""Host logic of bench.py's serving leg on the CPU, against a fake solve server.

serve_pass runs an open-loop Poisson schedule: arrivals beyond the in-flight cap are shed and counted,
completed requests are collected in submission order by a second thread, and latency runs from the
scheduled arrival.  The fake server completes each request after a fixed service time, so the
accounting can be checked exactly; a failed request must surface as an error after the collector
thread has been joined.
"""
import threading
import time
import types

import numpy as np
import pytest

import bench


class FakeServer:
    def __init__(self, service_s, fail_every=0):
        self.service_s = service_s
        self.fail_every = fail_every
        self.done = {}
        self.lock = threading.Lock()
        self.n = 0

    def submit(self, shape, alpha, k, f, u, tol, faces=None, field=0):
        with self.lock:
            self.n += 1
            rid = self.n
        t0 = time.perf_counter()
        status = -5 if self.fail_every and rid % self.fail_every == 0 else 0

        def finish():
            time.sleep(self.service_s)
            u[:1] = alpha
            self.done[rid] = {"status": status, "total_ms": 1e3 * (time.perf_counter() - t0),
                              "service_ms": 1e3 * self.service_s}
        threading.Thread(target=finish, daemon=True).start()
        return rid

    def wait(self, rid, timeout=-1.0):
        while rid not in self.done:
            time.sleep(1e-4)
        return self.done.pop(rid)


def _data():
    data, upool = {}, {}
    for gi, shp in enumerate(bench.SERVE_GRIDS):
        data[gi] = ([np.zeros(4), np.zeros(4)], None)
        upool[gi] = [np.zeros(4) for _ in range(bench.SERVE_CAP)]
    return data, upool


FAKE_BURA = types.SimpleNamespace(BURA_OK=0, BURA_ENOCONV=-5)


def test_light_load_serves_everything():
    data, upool = _data()
    out = bench.serve_pass(FAKE_BURA, np, None, FakeServer(0.002), data, upool, 200.0, 0.4, 0.1, 5)
    assert out["shed"] == 0 and out["completed"] == out["arrivals_measured"] > 40
    assert 2.0 <= out["p50_ms"] <= out["p99_ms"] < 200.0


def test_overload_sheds_beyond_the_cap():
    data, upool = _data()
    out = bench.serve_pass(FAKE_BURA, np, None, FakeServer(0.3), data, upool, 2000.0, 0.3, 0.05, 5)
    assert out["shed"] > 0
    assert out["completed"] + out["shed"] == out["arrivals_measured"]
    assert out["p99_ms"] >= 300.0


def test_a_failed_request_is_reported_after_the_join():
    data, upool = _data()
    before = threading.active_count()
    with pytest.raises(RuntimeError):
        bench.serve_pass(types.SimpleNamespace(BURA_OK=0, BURA_ENOCONV=-99), np, None, FakeServer(0.001, fail_every=3),
                         data, upool, 300.0, 0.2, 0.05, 7)
    time.sleep(0.05)
    assert threading.active_count() <= before + 2  # the collector has exited (fake completions may linger)
