"""Host logic of bench.py's CG side figure, with stand-ins for the binding and torch (no GPU): the
figure is assembled from the solver's outputs, and a failing solve is reported, not raised."""
import json
import os
import sys
import types

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class _Event:
    def __init__(self, **kw):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 2600.0


class _Torch:
    class cuda:
        Event = _Event

        @staticmethod
        def current_stream():
            return types.SimpleNamespace(cuda_stream=0)

        @staticmethod
        def synchronize():
            pass

    @staticmethod
    def from_numpy(a):
        class _T:
            def __init__(self, a):
                self.a = a

            def cuda(self):
                return self

            def clone(self):
                return _T(self.a.copy())
        return _T(a)


class _Ctx:
    def close(self):
        pass


class _Binding:
    HPSI_FP64 = 0

    def hpsi_gsphere(self, lattice, ecut, k):
        return np.zeros((1503, 3), dtype=np.int32)

    def hpsi_setup(self, *args):
        return _Ctx()

    def hpsi_kernel_stats(self, ctx, kernel, reset=False):
        return 4756, 0.0

    def cg_solve(self, ctx, ik, x, tol, maxiter):
        g = json.load(open(os.path.join(ROOT, "tests", "golden", "eigenvalues.json")))["c1"]["eigenvalues"][:16]
        return np.array(g) + 1e-13, 4740, np.full(16, 1e-9), 0


class _Failing(_Binding):
    def cg_solve(self, *args):
        raise RuntimeError("solver failed")


def test_cg_figure_from_solver_outputs():
    import bench
    out = bench.cg_throughput(_Binding(), _Torch())
    assert out["steps"] == 4740 and out["band_apps"] == 4756
    assert abs(out["band_apps_per_s"] - 4756 / 2.6) < 1e-9
    assert abs(out["max_eig_error_ha_vs_oracle"] - 1e-13) < 1e-14


def test_cg_figure_reports_failure():
    import bench
    out = bench.cg_throughput(_Failing(), _Torch())
    assert out == {"error": "solver failed"}
