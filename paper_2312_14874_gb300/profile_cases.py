"""One workload of the library, launched a few times: a target for a profiler.

    python -m paper_2312_14874_gb300.profile_cases seg_f32 [--reps 4]
    python -m paper_2312_14874_gb300.profile_cases scan_f32 [--reps 4]
    python -m paper_2312_14874_gb300.profile_cases compact_i32 [--reps 4]

seg_f32: the exclusive segmented scan of 20,000 segments with lengths
log-uniform in [1, 2^16] (116,893,251 fp32 elements, U[0,1)), through the
tuned variant (the partitioned kernel with the head bitmap).
scan_f32: the plain inclusive scan of the same 116,893,251 elements (tuned).
compact_i32: stream compaction of 2^28 int32 elements with half kept at random.
Every launch of the case's kernel is the same; the first ones warm the caches
and the module loads, so a profiler skips them.  Inputs are seeded and
synthetic; nothing is checked here (the test suite does that).
"""
import argparse
import sys

import torch

import paper_2312_14874_gb300 as gb
from paper_2312_14874_gb300 import _capi


def seg_f32(reps: int, dev: torch.device) -> None:
    import synth  # the seeded generators (repository root)
    off = synth.segment_offsets(20000, max_log2=16, seed=0)
    n = int(off[-1])
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    x = torch.rand(n, device=dev, generator=g)
    y = torch.empty_like(x)
    o = torch.from_numpy(off).to(dev)
    ws = gb.Workspace(gb.workspace_bytes(torch.float32, _capi.KIND_SEGMENTED, n, off.size - 1), dev)
    for _ in range(reps):
        gb.segmented(x, o, True, out=y, workspace=ws)
    torch.cuda.synchronize(dev)
    print(f"seg_f32: n={n}, segments={off.size - 1}, launches={reps}, status={gb.device_status(ws, dev)}")


def scan_f32(reps: int, dev: torch.device) -> None:
    n = 116893251
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    x = torch.rand(n, device=dev, generator=g)
    y = torch.empty_like(x)
    ws = gb.Workspace(gb.workspace_bytes(torch.float32, _capi.KIND_SCAN, n), dev)
    for _ in range(reps):
        gb.inclusive(x, out=y, workspace=ws)
    torch.cuda.synchronize(dev)
    print(f"scan_f32: n={n}, launches={reps}, status={gb.device_status(ws, dev)}")


def compact_i32(reps: int, dev: torch.device) -> None:
    n = 1 << 28
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    x = torch.randint(0, 1 << 30, (n,), dtype=torch.int32, device=dev, generator=g)
    flags = (torch.rand(n, device=dev, generator=g) < 0.5).view(torch.uint8)
    y = torch.empty_like(x)
    ws = gb.Workspace(gb.workspace_bytes(torch.int32, _capi.KIND_COMPACT, n), dev)
    count = None
    for _ in range(reps):
        _, count = gb.compact(x, flags, out=y, workspace=ws)
    torch.cuda.synchronize(dev)
    print(f"compact_i32: n={n}, kept={int(count.item())}, launches={reps}, status={gb.device_status(ws, dev)}")


CASES = {"seg_f32": seg_f32, "scan_f32": scan_f32, "compact_i32": compact_i32}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--reps", type=int, default=4)
    args = ap.parse_args(argv)
    if not torch.cuda.is_available():
        print("a CUDA device is needed", file=sys.stderr)
        return 2
    CASES[args.case](args.reps, torch.device("cuda", 0))
    return 0


if __name__ == "__main__":
    sys.exit(main())
