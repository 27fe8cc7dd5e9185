"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1506_04694_gb300 as pk
    pk.build.build()
    return torch, pk
