"""Host logic of the autograd backward's workspace (no GPU needed): the
worst-case workspace (no map can overflow it, so the backward reads no
status) when it fits the byte budget and half the free memory, else the
default size, grown to the reported record count after an overflow."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture()
def ws_env(monkeypatch):
    from paper_2604_21984_gb300 import autograd, build, capi
    build.build()
    made = []

    def fake_workspace(H, W, K, cap, max_records=0, device="cuda"):
        made.append(max_records)
        return ("ws", max_records)
    free = {"bytes": 64 << 30}
    monkeypatch.setattr(capi, "backward_workspace", fake_workspace)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda device=None: (free["bytes"], 96 << 30))
    monkeypatch.setattr(autograd, "_WS", autograd._Workspaces())
    return autograd, capi, made, free


def test_worst_case_workspace_when_it_fits(ws_env):
    autograd, capi, made, _ = ws_env
    H = W = 2048
    K, N = 16, 262144
    worst = capi.sad_backward_max_records(H, W, K, N)
    assert worst == (H // 16) * (W // 16) * min(256 * K, N)
    nbytes = capi.lib().sad_backward_workspace_bytes(H, W, K, N, worst)
    assert nbytes <= autograd.WORST_CASE_BYTES          # about 4 GB: inside the 8 GiB budget
    ws, exact = autograd._WS.get("cuda:0", H, W, K, N)
    assert exact and made == [worst]
    # cached: the same problem allocates nothing new
    assert autograd._WS.get("cuda:0", H, W, K, N) == (ws, True) and made == [worst]


def test_default_workspace_and_regrow_when_over_budget(ws_env, monkeypatch):
    autograd, capi, made, _ = ws_env
    monkeypatch.setattr(autograd, "WORST_CASE_BYTES", 1 << 20)
    H = W = 512
    K, N = 16, 16384
    ws, exact = autograd._WS.get("cuda:0", H, W, K, N)
    assert not exact and made == [0]                    # the default size
    # an overflow reported 123456 records: the workspace grows to that count
    ws2, exact2 = autograd._WS.get("cuda:0", H, W, K, N, min_records=123456)
    assert not exact2 and made == [0, 123456]
    # a smaller later request keeps the grown workspace
    assert autograd._WS.get("cuda:0", H, W, K, N, min_records=1000) == (ws2, False)
    assert made == [0, 123456]


def test_default_workspace_when_free_memory_is_short(ws_env):
    autograd, capi, made, free = ws_env
    H = W = 2048
    K, N = 16, 262144
    nbytes = capi.lib().sad_backward_workspace_bytes(H, W, K, N, capi.sad_backward_max_records(H, W, K, N))
    free["bytes"] = 2 * nbytes - 1                      # half of it is just too little
    _, exact = autograd._WS.get("cuda:0", H, W, K, N)
    assert not exact and made == [0]
