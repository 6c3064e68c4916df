"""bmpc_create_batch_static: solving without a caller-supplied scratch arena.

Callers that cannot allocate device memory for the solver (real-time control loops that
forbid allocation while running, plug-ins whose framework owns all device buffers) create
the batch with bmpc_create_batch_static; the solver scratch is then the library's fixed
16 MiB device array.  Through the C ABI, two solves in a row on such a batch must give the
same results as the regular entry point bit for bit (the same kernel, block size and inputs, so
the same arithmetic), with a solve of a different batch through the same array in between (stale
scratch from it would show), and a batch that needs more scratch than the array holds must be
refused.
"""
import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problems():
    return [scenes.config1(2), scenes.config2(3)] + scenes.config4(4, 5)


def _same(a, b):
    for key in ("x", "u", "lam", "y"):
        assert np.array_equal(b[key], a[key]), key
    for key in ("status", "inner_iters", "outer_iters", "ls_evals"):
        assert a[key] == b[key], key


def test_static_scratch_matches_regular_entry_point_twice():
    from paper_2506_13624_b300 import bmpc
    ps = _problems()
    opts = bmpc.default_opts(block_threads=64)
    ref = bmpc.Batch(ps)
    ref.set_problems()
    ref.solve(opts)
    want = ref.get_solutions()
    ref.close()

    sb = bmpc.StaticScratchBatch(ps)
    assert sb.scratch_bytes <= bmpc.STATIC_SCRATCH_BYTES
    sb.set_problems()
    for call in range(2):
        sb.solve(opts)
        got = sb.get_solutions()
        for a, b in zip(want, got):
            _same(a, b)
        if call == 0:
            # another batch through the shared array leaves its own data there
            other = bmpc.StaticScratchBatch(scenes.config4(9, 6) + [scenes.config2(11)])
            other.set_problems()
            other.solve(opts)
            assert all(r["inner_iters"] > 0 for r in other.get_solutions(want_arrays=False))
            other.close()
    sb.close()
    assert sum(r["status"] == 0 for r in want) >= len(ps) - 1


def test_static_scratch_refuses_oversized_batches():
    from paper_2506_13624_b300 import bmpc
    ps = [scenes.config3(0)] * 12          # about 19 MB of scratch: more than the 16 MiB array
    with pytest.raises(RuntimeError) as e:
        bmpc.StaticScratchBatch(ps)
    assert str(bmpc.ERR_SPACE) in str(e.value)
