"""nrrs_split_noalloc against nrrs_split, through the C ABI (GPU).

nrrs_split_noalloc serves callers that cannot allocate device memory on the call path
(an engine whose device memory all belongs to its own arena, or a frame loop that
cannot take the device-wide stall cudaMalloc / cudaFree may cause).  It must give the
same results as nrrs_split -- bit for bit, the bar for this integer work -- on two calls
in a row, since every call reuses the one scratch array inside the library.
"""
import numpy as np
import pytest

from paper_2510_07868_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    q = I.random_q(n, seed=seed, scale=3.0)
    pix = np.sort(rng.integers(0, max(1, n // 4), n)).astype(np.int32)
    smp = rng.integers(0, 16, n).astype(np.int32)
    lin = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32).view(np.int32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    return dev(q), dev(pix), dev(smp), dev(lin)


def _empty_inputs():
    z = lambda dt: torch.zeros(1, dtype=dt, device="cuda")  # noqa: E731
    return z(torch.float32), z(torch.int32), z(torch.int32), z(torch.int32)


def _outputs(n, cap):
    return (torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda"),
            torch.full((max(n, 1),), -7, dtype=torch.int64, device="cuda"),
            torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda"),
            torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda"),
            torch.full((1,), -7, dtype=torch.int64, device="cuda"),
            torch.full((1,), -7, dtype=torch.int64, device="cuda"))


def _run(nrrs, fn, ins, n, F, depth, frame, cap):
    q, pix, smp, lin = ins
    X, prefix, cp, cl, tot, drop = _outputs(n, cap)
    dF = torch.tensor([F], dtype=torch.float32, device="cuda")
    args = (q, n, dF, pix, smp, lin, depth, 11, 5, frame, cap, X, prefix, cp, cl, tot, drop)
    if fn == "split":
        nrrs.nrrs_split(None, *args)
    else:
        nrrs.nrrs_split_noalloc(*args)
    torch.cuda.synchronize()
    S = int(tot.item())
    m = min(S, cap)
    return (X[:n].cpu().numpy(), prefix[:n].cpu().numpy(), cp[:m].cpu().numpy(),
            cl[:m].cpu().numpy(), S, int(drop.item()))


def test_noalloc_matches_split_on_two_calls_in_a_row():
    from paper_2510_07868_b300 import nrrs

    assert torch.cuda.is_available()
    cases = [(300_001, 0.6, 3, 1, 2), (70_000, 1.0, 7, 2, 0.5)]  # second one overflows
    for n, F, depth, frame, capmul in cases:
        ins = _inputs(n, seed=n)
        cap = int(capmul * n)
        ref = _run(nrrs, "split", ins, n, F, depth, frame, cap)
        got = _run(nrrs, "noalloc", ins, n, F, depth, frame, cap)
        for a, b in zip(ref[:4], got[:4]):
            np.testing.assert_array_equal(a, b)
        assert ref[4:] == got[4:]
    assert got[5] > 0  # the second call dropped children at the capacity


@pytest.mark.parametrize("n", [0, 1, 255, 4095, 4096, 4097])
def test_noalloc_matches_split_at_chunk_edges(n):
    """Sizes where the no-allocation variant's grid (one block per 4096 parents) leaves a
    block with no tile or a one-parent tail, while nrrs_split spreads the same parents
    over its fixed grid: both must agree bit for bit."""
    from paper_2510_07868_b300 import nrrs

    for call in range(2):
        ins = _inputs(n, seed=n + 17 * call) if n else _empty_inputs()
        cap = 2 * n + 8
        ref = _run(nrrs, "split", ins, n, 0.8, 2 + call, call, cap)
        got = _run(nrrs, "noalloc", ins, n, 0.8, 2 + call, call, cap)
        for a, b in zip(ref[:4], got[:4]):
            np.testing.assert_array_equal(a, b)
        assert ref[4:] == got[4:]


def test_noalloc_block_counts_beyond_32_bits():
    """4096 parents in one block, each asking for about 2^23 children: the block's count
    passes 2^32 and must not saturate (the totals and prefixes equal nrrs_split's)."""
    from paper_2510_07868_b300 import nrrs

    n = 4096
    rng = np.random.default_rng(23)
    q = torch.from_numpy((8388607.5 - rng.integers(0, 64, n) * 0.5).astype(np.float32)).cuda()
    _, pix, smp, lin = _inputs(n, seed=23)
    cap = 1 << 20
    ref = _run(nrrs, "split", (q, pix, smp, lin), n, 1.0, 4, 1, cap)
    got = _run(nrrs, "noalloc", (q, pix, smp, lin), n, 1.0, 4, 1, cap)
    assert ref[4] > 2**32
    for a, b in zip(ref[:4], got[:4]):
        np.testing.assert_array_equal(a, b)
    assert ref[4:] == got[4:]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2510_07868_b300 import nrrs

    ins = _inputs(16, seed=1)
    X, prefix, cp, cl, tot, drop = _outputs(16, 32)
    dF = torch.ones(1, dtype=torch.float32, device="cuda")
    with pytest.raises(nrrs.NrrsError) as e:
        nrrs.nrrs_split_noalloc(ins[0], 67_108_865, dF, ins[1], ins[2], ins[3], 1, 1, 0, 0, 32, X,
                                prefix, cp, cl, tot, drop)
    assert e.value.code == 1 and "67108864" in str(e.value)
    # nothing was launched: the outputs still hold their fill value
    torch.cuda.synchronize()
    assert int(tot.item()) == -7
