"""The C-ABI library builds, loads and exports every symbol include/warpsci.h declares;
host-side validation paths that need no GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2408_00930_gb300 import warpsci as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "warpsci.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ws_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_00930_gb300 import build
    build.build()
    return W.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "ws_create" in names and "ws_rollout" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(W.EXPORTED) | set(n for n in names if n not in W.EXPORTED)


@pytest.mark.parametrize("struct", ["ws_config", "ws_request", "ws_server_stats", "ws_launch"])
def test_struct_layout_matches_header(lib, tmp_path, struct):
    """Each ctypes mirror has the C compiler's size and field offsets."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    cls = getattr(W, struct)
    fields = [f for f, _ in cls._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "warpsci.h"\nint main(void){\n'
                   f'printf("%zu\\n", sizeof({struct}));\n' +
                   "".join(f'printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields) +
                   "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                            check=True).stdout.split()]
    assert vals[0] == C.sizeof(cls)
    for f, off in zip(fields, vals[1:]):
        assert getattr(cls, f).offset == off, f


def test_query_bytes_validation(lib):
    cfg, _ = W.make_config(W.WS_ENV_CONTROL, W.WS_PATH_PLAIN_FP32, 1000, 200, 200, 64, 64)
    st, sb, rb, ns = W.ws_query_bytes(cfg)
    assert st == W.WS_OK and ns == 1000 and sb > 0 and rb >= 200 * 1000 * (16 + 4 * 4 + 1)
    bad, _ = W.make_config(W.WS_ENV_CONTROL, W.WS_PATH_PLAIN_FP32, 0, 200, 200, 64, 64)
    assert W.ws_query_bytes(bad)[0] == W.WS_ERR_INVALID
    bad, _ = W.make_config(W.WS_ENV_LANDSCAPE, W.WS_PATH_PLAIN_FP32, 8, 10, 10, 16, 16, dim=0,
                           n_gauss=4)
    assert W.ws_query_bytes(bad)[0] == W.WS_ERR_INVALID
    cfg.struct_size = 8
    assert W.ws_query_bytes(cfg)[0] == W.WS_ERR_INVALID
    # the energy target is a landscape option and must be finite
    ok, _ = W.make_config(W.WS_ENV_LANDSCAPE, W.WS_PATH_PLAIN_FP32, 8, 10, 10, 16, 16, dim=4,
                          n_gauss=4, energy_target=-0.5)
    assert ok.flags & W.WS_FLAG_ENERGY_TARGET and W.ws_query_bytes(ok)[0] == W.WS_OK
    ok.energy_target = float("nan")
    assert W.ws_query_bytes(ok)[0] == W.WS_ERR_INVALID
    bad, _ = W.make_config(W.WS_ENV_CONTROL, W.WS_PATH_PLAIN_FP32, 8, 10, 10, 16, 16,
                           energy_target=-0.5)
    assert W.ws_query_bytes(bad)[0] == W.WS_ERR_INVALID
    bad.flags = 4
    assert W.ws_query_bytes(bad)[0] == W.WS_ERR_INVALID


def test_economy_slot_count_uses_agent_counts(lib):
    import oracle
    cfg, keep = W.make_config(W.WS_ENV_ECONOMY, W.WS_PATH_PLAIN_FP32, 3, 10, 540, 128, 128,
                              agents_per_env=[8, 100, 256])
    assert W.ws_query_bytes(cfg)[3] == 8 + 100 + 256 + 3
    cfg, _ = W.make_config(W.WS_ENV_ECONOMY, W.WS_PATH_PLAIN_FP32, 50, 10, 540, 128, 128,
                           param_seed=77)
    # counts drawn on the host by the library equal the oracle's draws
    exp = sum(oracle.econ_agent_count(77, e) for e in range(50)) + 50
    assert W.ws_query_bytes(cfg)[3] == exp
    bad, _ = W.make_config(W.WS_ENV_ECONOMY, W.WS_PATH_PLAIN_FP32, 2, 10, 540, 128, 128,
                           agents_per_env=[1, 5])
    assert W.ws_query_bytes(bad)[0] == W.WS_ERR_INVALID


def test_create_rejects_small_or_null_buffers(lib):
    cfg, _ = W.make_config(W.WS_ENV_CONTROL, W.WS_PATH_PLAIN_FP32, 10, 4, 200, 8, 8)
    st, ctx = W.ws_create(cfg, None, 0, None, 0, None)
    assert st == W.WS_ERR_INVALID and ctx is None
    st, sb, rb, _ = W.ws_query_bytes(cfg)
    st, ctx = W.ws_create(cfg, 256, sb - 1, 512, rb, None)   # never dereferenced
    assert st == W.WS_ERR_NOMEM and ctx is None
    st, ctx = W.ws_create(cfg, 257, sb, 512, rb, None)
    assert st == W.WS_ERR_INVALID and ctx is None


def test_null_context_calls(lib):
    assert lib.ws_step(None) == W.WS_ERR_INVALID
    assert lib.ws_rollout(None, 3) == W.WS_ERR_INVALID
    assert lib.ws_sync(None, 1) == W.WS_ERR_INVALID
    assert W.ws_last_error(None) == "null context"
    W.ws_destroy(None)
