"""Runs bench.main() on the CPU with the CUDA library, CUDA events and
streams and the process group replaced by fakes, so that the shape of the
JSON line bench.py prints can be checked without a GPU.  The numbers are
the fakes' (every timed region reads 2 ms, every kernel-timing hook 0.2 /
0.01 / 1.9 / 0.05 ms); the CPU oracle baseline is real.

Run as a separate process (it patches torch): python tests/bench_fakes.py
[bench arguments...].
"""
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import bench  # noqa: E402
import paper_1203_5128_gb300 as bf  # noqa: E402
import paper_1203_5128_gb300.replicas as replicas  # noqa: E402

EVENT_MS = 2.0
KERNEL_MS = [0.2, 0.01, 1.9, 0.05]


class FakeEvent:
    def __init__(self, *a, **k):
        pass

    def record(self, *a):
        pass

    def elapsed_time(self, other):
        return EVENT_MS


class FakeStream:
    cuda_stream = 0

    def wait_event(self, ev):
        pass


class FakeReplicas:
    def __init__(self, *a):
        pass

    def barrier(self):
        pass

    def max(self, x):
        return x

    def close(self):
        pass


class FakePlan:
    def __init__(self, H, W, sigma_s, sigma_r, eps, **kw):
        self.H, self.W = H, W
        self.R = int(sigma_s) if kw.get("spatial") == "box" else int(np.ceil(3 * sigma_s))
        t = kw.get("t_tile", 64)
        self.N = 17
        self.n_sets = (-(-H // t)) * (-(-W // t)) if kw.get("t_mode") == "tile" else 1

    def close(self):
        pass


def install():
    torch.cuda.Event = FakeEvent
    torch.cuda.Stream = FakeStream
    torch.cuda.current_stream = lambda *a: FakeStream()
    torch.cuda.synchronize = lambda *a: None
    torch.cuda.set_device = lambda *a: None
    torch.cuda.current_device = lambda: 0
    torch.cuda.get_device_properties = lambda d: types.SimpleNamespace(multi_processor_count=152)
    torch.Tensor.cuda = lambda self, *a, **k: self
    torch.Tensor.pin_memory = lambda self, *a, **k: self
    empty = torch.empty
    torch.empty = lambda *a, **k: empty(*a, **{n: v for n, v in k.items() if n != "device"})
    replicas.Replicas = FakeReplicas
    bench.ClockSampler = lambda *a: types.SimpleNamespace(
        start=lambda: None,
        stop=lambda: {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 1})
    bf.bf_plan = lambda *a, **k: FakePlan(*a, **k)
    bf.bf_execute = lambda plan, f, out=None, stream=None: out
    bf.bf_execute_batch = lambda plans, fs, outs=None, stream=None: outs
    bf.bf_backward = lambda *a, **k: None
    bf.bf_execute_host = lambda *a, **k: None
    bf.bf_set_timing = lambda *a: None
    bf.bf_get_timing = lambda plan: (list(KERNEL_MS), 1)
    bf.bf_get_info = lambda p: types.SimpleNamespace(R=p.R, N=264, M=94, K=77, H=p.H, W=p.W,
                                                     n_sets=p.n_sets, n_rechecked=0,
                                                     n_guarded=0, terms_total=77)
    bf.bf_get_sets = lambda p: (np.full(p.n_sets, 200.0, np.float32),
                                np.full(p.n_sets, 200, np.int32), np.full(p.n_sets, 60, np.int32))


if __name__ == "__main__":
    install()
    sys.argv = ["bench.py"] + sys.argv[1:]
    bench.main()
