"""The allocation-free entry point (for callers that cannot allocate device
memory) against the allocating entry point: same operation, same inputs,
identical bits, on several calls in a row through the one shared work area."""
import random

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _limbs(v, n):
    return np.frombuffer(v.to_bytes(4 * n, "little"), dtype=np.uint32).copy()


def test_noalloc_matches_allocating_entry_point():
    import torch
    from paper_0902_0852_gb300 import build, hk
    build.build()
    hk.lib()
    stream = torch.cuda.current_stream()
    rng = random.Random(7)

    def dev(a):
        return torch.from_numpy(a.view(np.int32)).cuda()

    cases = []
    for L in (64, 256, 768):
        P = 32 * L
        a = rng.getrandbits(P) | (1 << (P - 1))
        b = rng.getrandbits(P) | (1 << (P - 1))
        cases.append((3, L, a, -5, b, 11))          # correctly rounded division
        cases.append((2, L, a, 7, None, 0))         # correctly rounded square root
        cases.append((3, L, b, 2, a, -3))           # division again, new operands
    cases.append((1, 96, (1 << 3071) | 12345, 0, None, 0))          # reciprocal floor
    cases.append((0, 1, rng.getrandbits(5000), 0, rng.getrandbits(3000), 0))  # product
    cases.append((4, 128, rng.getrandbits(9000) | 1, -40, None, 0))  # rounding
    for op, L, x, ex, y, ey in cases:
        want = hk.hk_selftest_mp(op, L, x, ex=ex, y=y, ey=ey)
        nx = L if op in (1, 2, 3) else max(1, (x.bit_length() + 31) // 32)
        ny = 0 if y is None else (L if op == 3 else max(1, (y.bit_length() + 31) // 32))
        nout = {0: nx + ny + 2, 1: L + 2}.get(op, L)
        xd = dev(_limbs(x, nx))
        yd = dev(_limbs(y, ny)) if y is not None else None
        # dirty output buffers (all ones): the result must not depend on
        # what the caller's memory held before the call
        out = torch.full((nout,), -1, dtype=torch.int32, device="cuda")
        eo = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        hk.hk_mp_op_noalloc(op, L, xd, ex, yd, ey, out, eo, stream)
        torch.cuda.synchronize()
        val = int.from_bytes(out.cpu().numpy().view(np.uint32).tobytes(), "little")
        e = eo.cpu().tolist()
        assert e[1] == 0
        got = val if op in (0, 1) else (val, e[0])
        assert got == want, (op, L)


def test_noalloc_rejects_oversized_requests():
    import torch
    from paper_0902_0852_gb300 import build, hk
    build.build()
    x = torch.zeros(4000, dtype=torch.int32, device="cuda")
    y = torch.zeros(200, dtype=torch.int32, device="cuda")
    out = torch.zeros(4300, dtype=torch.int32, device="cuda")
    eo = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(hk.HKError) as ei:
        hk.hk_mp_op_noalloc(0, 1, x, 0, y, 0, out, eo)
    assert ei.value.code == hk.HK_ERR_ARG
    # rounded operations are limited to P = 32 L <= 32768 bits: L = 1025 is
    # refused although nx + ny + L stays within the work area
    for op, L, nx, ny in [(1, 1025, 1025, 0), (2, 1025, 1025, 0), (3, 1025, 1025, 1025), (4, 1025, 8, 0)]:
        with pytest.raises(hk.HKError) as ei:
            hk.hk_mp_op_noalloc(op, L, x[:nx], 0, None if ny == 0 else x[:ny], 0, out, eo)
        assert ei.value.code == hk.HK_ERR_ARG, (op, L)
