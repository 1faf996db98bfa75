"""Helpers shared by the GPU tests (no method arithmetic here)."""
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


_ctx = None


def ctx():
    global _ctx
    need_gpu()
    import paper_2301_04642_gb300 as fe
    if _ctx is None:
        _ctx = fe.Context(device=0)
    return _ctx
