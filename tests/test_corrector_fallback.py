"""The corrector's fallback policy (corrector.infer(..., fallback=True)), on the host: with
the library calls replaced by fakes, a clear status word returns the corrector's output and
any other status returns the uncorrected input, with a warning.  The kernels themselves and
their status word are covered by the GPU tests."""
import pytest
import torch

from paper_2007_06289_gb300 import corrector


@pytest.fixture()
def fake_lib(monkeypatch):
    state = {"status": 0, "calls": 0}

    def forward(params, x, y, ws, train=False, stream=None):
        state["calls"] += 1
        y.copy_(x + 1.0)                     # a stand-in "correction"

    def last_error():
        s, state["status"] = state["status"], 0   # read and clear, like the library
        return s

    monkeypatch.setattr(corrector.fbp, "fbp_cnn_forward", forward)
    monkeypatch.setattr(corrector.fbp, "fbp_cnn_last_error", last_error)
    monkeypatch.setattr(corrector.fbp, "fbp_cnn_workspace_bytes", lambda N, B, train: 16)
    monkeypatch.setattr(corrector.fbp, "fbp_status_str", lambda s: "bounded wait timed out")
    return state


def test_clear_status_returns_the_correction(fake_lib):
    x = torch.arange(32.0).reshape(2, 4, 4)
    y = corrector.infer(torch.zeros(3), x, fallback=True)
    assert torch.equal(y, x + 1.0) and fake_lib["calls"] == 1


def test_failed_status_returns_the_uncorrected_input(fake_lib):
    x = torch.arange(32.0).reshape(2, 4, 4)
    fake_lib["status"] = 6                   # FBP_ERR_TIMEOUT
    with pytest.warns(RuntimeWarning, match="uncorrected"):
        y = corrector.infer(torch.zeros(3), x, fallback=True)
    assert torch.equal(y, x) and y.data_ptr() != x.data_ptr()
    assert fake_lib["status"] == 0           # the read cleared it


def test_without_fallback_the_status_is_not_read(fake_lib):
    x = torch.ones(1, 4, 4)
    fake_lib["status"] = 6
    y = corrector.infer(torch.zeros(3), x)
    assert torch.equal(y, x + 1.0) and fake_lib["status"] == 6
