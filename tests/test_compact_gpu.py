"""GPU parity for stream compaction (the scan of keep flags fused with the
gather), through the C ABI, against the CPU oracle: bit-exact outputs and
counts for every variant, flag densities from none to all, ragged tails,
misaligned flag and payload pointers (element-wise loads), bool flags, and
many 16-tile chunks in a child process."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2312_14874_gb300 as gb
from paper_2312_14874_gb300 import _capi

pytestmark = pytest.mark.gpu

SIZES = [1, 3, 5119, 5120, 5121, 3 * 5120 * 7 + 13, 1_000_003]


def dev():
    return torch.device("cuda", 0)


def flags_of(n, density, seed):
    u = synth.unit_f32(n, seed=seed)
    return (u < density).astype(np.uint8) * (1 + synth.uniform_i32(n, 200, seed=seed + 1)).astype(np.uint8)


@pytest.mark.parametrize("key", ["i32", "f32"])
@pytest.mark.parametrize("density", [0.0, 0.02, 0.5, 1.0])
def test_compact_sizes_and_densities(key, density):
    for n in SIZES:
        a = synth.uniform_i32(n, 1 << 31, seed=n % 97) if key == "i32" else synth.normal_f32(n, seed=n % 97)
        f = flags_of(n, density, seed=n % 89)
        want = oracle.compact(a, f)
        x, fl = torch.from_numpy(a).to(dev()), torch.from_numpy(f).to(dev())
        for v in range(gb.num_variants(torch.int32, _capi.KIND_COMPACT)):
            out, cnt = gb.compact(x, fl, variant=v)
            k = int(cnt.item())
            assert k == want.size, (n, v, k, want.size)
            assert np.array_equal(out[:k].cpu().numpy().view(np.uint32), want.view(np.uint32)), (n, v)
    assert gb.device_status() == 0


def test_compact_misaligned_and_bool_flags():
    """Every variant (the partitioned and the single-pass compaction) on a
    payload and flags at odd offsets (element-wise loads), bool flags, and an
    output at an odd offset between guard words."""
    n = 4 * 5120 + 77
    a = synth.uniform_i32(n + 1, 1 << 30, seed=4)
    f = flags_of(n + 1, 0.3, seed=5)
    xa = torch.from_numpy(a).to(dev())
    fa = torch.from_numpy(f).to(dev())
    for v in range(gb.num_variants(torch.int32, _capi.KIND_COMPACT)):
        # payload at an element offset (not 16-byte aligned), flags at a byte offset
        x, fl = xa[1:], fa[1:]
        out, cnt = gb.compact(x, fl, variant=v)
        want = oracle.compact(a[1:], f[1:])
        assert int(cnt.item()) == want.size, v
        assert np.array_equal(out[:want.size].cpu().numpy(), want), v
        out, cnt = gb.compact(xa[:n], fa[:n] != 0, variant=v)  # bool flags
        want = oracle.compact(a[:n], f[:n])
        assert int(cnt.item()) == want.size and np.array_equal(out[:want.size].cpu().numpy(), want), v
        # output at an element offset (not 16-byte aligned): the runs leave with
        # single-element stores; the guard words around it stay untouched
        ob = torch.full((n + 2,), -7, dtype=torch.int32, device=dev())
        out, cnt = gb.compact(xa[:n], fa[:n], out=ob[1:n + 1], variant=v)
        k = int(cnt.item())
        assert k == want.size and np.array_equal(out[:k].cpu().numpy(), want), v
        assert int(ob[0].item()) == -7 and int(ob[n + 1].item()) == -7, v
    assert gb.device_status() == 0


def test_compact_abi_errors():
    L = _capi.lib()
    n = 1000
    x = torch.zeros(n, dtype=torch.int32, device=dev())
    fl = torch.ones(n, dtype=torch.uint8, device=dev())
    y = torch.empty_like(x)
    cnt = torch.full((2,), 7, dtype=torch.int64, device=dev())
    ws = gb.Workspace(gb.workspace_bytes(torch.int32, _capi.KIND_COMPACT, n))
    s = torch.cuda.current_stream().cuda_stream
    args = (ws.ptr, ws.nbytes, 0, s)
    assert L.compact_i32(x.data_ptr(), fl.data_ptr(), x.data_ptr(), n, cnt.data_ptr(), *args) == \
        _capi.ERR_INVALID_ARG  # in place
    assert L.compact_i32(x.data_ptr(), None, y.data_ptr(), n, cnt.data_ptr(), *args) == _capi.ERR_INVALID_ARG
    assert L.compact_i32(x.data_ptr(), fl.data_ptr(), y.data_ptr(), n, None, *args) == _capi.ERR_INVALID_ARG
    assert L.compact_i32(x.data_ptr(), fl.data_ptr(), y.data_ptr(), -1, cnt.data_ptr(), *args) == \
        _capi.ERR_INVALID_ARG
    assert L.compact_i32(x.data_ptr(), fl.data_ptr(), y.data_ptr(), n, cnt.data_ptr() + 4, *args) == \
        _capi.ERR_ALIGNMENT
    # n = 0 writes a zero count
    assert L.compact_i32(None, None, None, 0, cnt.data_ptr(), *args) == _capi.OK
    torch.cuda.synchronize()
    assert int(cnt[0].item()) == 0
    assert gb.device_status(ws) == 0


COMPACT_CHUNK_SCRIPT = r"""
import sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import oracle, synth
import paper_2312_14874_gb300 as gb
dev = torch.device("cuda", 0)
n = 16 * 5120 * 23 + 611
a = synth.uniform_i32(n, 1 << 31, seed=11)
for density in (0.001, 0.5, 0.97):
    f = (synth.unit_f32(n, seed=12) < density).astype(np.uint8)
    want = oracle.compact(a, f)
    x, fl = torch.from_numpy(a).to(dev), torch.from_numpy(f).to(dev)
    for v in range(2):
        out, cnt = gb.compact(x, fl, variant=v)
        k = int(cnt.item())
        assert k == want.size and np.array_equal(out[:k].cpu().numpy(), want), (density, v)
assert gb.device_status() == 0
print("ok")
"""


@pytest.mark.parametrize("lag", [1, 3])
def test_compact_small_chunks(tmp_path, lag):
    """16-tile chunks (child process): chunk scans of the keep counts, chained
    chunk prefixes and the total written by the last chunk."""
    import os
    import subprocess
    import sys
    from conftest import ROOT
    script = tmp_path / "compact.py"
    script.write_text(COMPACT_CHUNK_SCRIPT)
    env = dict(os.environ, GBSCAN_CHUNK_BYTES="4096", GBSCAN_CHUNK_LAG=str(lag))
    r = subprocess.run([sys.executable, str(script), ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
