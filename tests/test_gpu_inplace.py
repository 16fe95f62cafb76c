"""In-place mode: the digit passes permute the keys inside the caller's
buffer (shared-memory pass for small buckets, block permutation for large
ones).  Results must equal the oracle's (and the ping-pong mode's) bit for
bit; the auxiliary bytes are reported and stay below the ping-pong
workspace."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import assert_bit_exact, check_full_size, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2603_08929_gb300 import build as b
    b.build()
    torch.cuda.set_device(0)


def sort_inplace(x, descending=False):
    import torch
    import paper_2603_08929_gb300 as bs
    t = to_device(x)
    h = bs.Handle()
    ws = torch.empty(max(1, bs.workspace_bytes(t.numel(), x.dtype.name, mode=bs.MODE_INPLACE)),
                     dtype=torch.uint8, device=t.device)
    bs.bsort_keys_ws(h, t, ws, descending=descending, mode=bs.MODE_INPLACE)
    assert h.get_error() == 0
    aux = h.last_aux_bytes()
    return t.cpu().numpy(), aux


# sizes: one finish unit, shared-memory buckets only, one block-permuted level
# then units, two block-permuted levels, ragged
SIZES = [3000, 40000, 300001, 1 << 20, (1 << 22) + 7]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("dtype", ["int32", "uint32", "float32", "int64", "uint64", "float64"])
def test_inplace_uniform(dtype, n):
    if n > 1 << 21 and dtype not in ("int32", "float64"):
        pytest.skip("large sizes: one 4- and one 8-byte type")
    x = W.make("uniform", dtype, n, seed=n % 1000)
    got, aux = sort_inplace(x)
    assert_bit_exact(got, O.bsort(x.copy()), "%s n=%d" % (dtype, n))


@pytest.mark.parametrize("dist", ["zipf", "normal", "distinct8", "sorted", "reverse"])
@pytest.mark.parametrize("dtype", ["int32", "float64"])
def test_inplace_distributions(dtype, dist):
    n = 700001
    x = W.make(dist, dtype, n, seed=3)
    got, _ = sort_inplace(x)
    assert_bit_exact(got, O.bsort(x.copy()), "%s %s" % (dtype, dist))


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_inplace_float_edge_descending(dtype):
    x = W.make("float_edge", dtype, 500003, seed=9)
    got, _ = sort_inplace(x, descending=True)
    assert_bit_exact(got, O.bsort(x.copy(), descending=True), dtype)


@pytest.mark.parametrize("dtype", ["uint8", "int16", "float16"])
def test_inplace_counting_dtypes(dtype):
    x = W.make("uniform", dtype, 100003, seed=4)
    got, aux = sort_inplace(x)
    assert_bit_exact(got, O.bsort(x.copy()), dtype)


def test_inplace_equals_pingpong_and_reports_aux():
    import torch
    import paper_2603_08929_gb300 as bs
    n = 1 << 24
    x = W.make("uniform", "int32", n, seed=21)
    got, aux = sort_inplace(x)
    t = to_device(x)
    h = bs.Handle()
    ws = torch.empty(bs.workspace_bytes(n, "int32"), dtype=torch.uint8, device=t.device)
    bs.bsort_keys_ws(h, t, ws)
    pp_aux = h.last_aux_bytes()
    assert_bit_exact(got, t.cpu().numpy(), "in-place vs ping-pong")
    reserved = bs.workspace_bytes(n, "int32", mode=bs.MODE_INPLACE)
    assert 0 < aux <= reserved < pp_aux
    # 2^24 keys: the second level's 65536-key buckets are just above the
    # shared-memory pass, the worst case for block buffers; still well below
    # the ping-pong mode's second copy of the keys
    assert aux < 0.5 * n * 4, aux / (n * 4)


def test_inplace_full_size():
    n = 1 << 26
    x = W.make("uniform", "int32", n, seed=22)
    got, aux = sort_inplace(x)
    check_full_size(x, got, False)


def test_bounded_wait_times_out_and_context_survives():
    """The library's one kind of device wait, on a flag nothing sets, gives up
    and reports BSORT_ERR_TIMEOUT; the next sort on the same context works."""
    import paper_2603_08929_gb300 as bs
    assert bs.selftest_bounded_wait() == 7
    x = W.make("uniform", "int32", 1 << 20, seed=8)
    got, _ = sort_inplace(x)
    assert_bit_exact(got, O.bsort(x.copy()), "after the timed-out wait")


@pytest.mark.parametrize("dtype", ["int32", "float64"])
def test_inplace_unaligned_view(dtype):
    """A view one key past a 16-byte boundary: scalar paths everywhere."""
    import torch
    import paper_2603_08929_gb300 as bs
    n = 700003
    x = W.make("uniform", dtype, n + 1, seed=9)
    base = to_device(x)
    t = base[1:]
    h = bs.Handle()
    ws = torch.empty(bs.workspace_bytes(n, dtype, mode=bs.MODE_INPLACE), dtype=torch.uint8, device=t.device)
    bs.bsort_keys_ws(h, t, ws, mode=bs.MODE_INPLACE)
    assert h.get_error() == 0
    out = base.cpu().numpy()
    assert_bit_exact(out[1:], O.bsort(x[1:].copy()), "unaligned in-place")
    assert out[:1].view(np.uint8).tobytes() == x[:1].view(np.uint8).tobytes()  # the key before the view is untouched


@pytest.mark.parametrize("mode", ["pingpong", "inplace"])
def test_python_sort_modes(mode):
    import paper_2603_08929_gb300 as bs
    x = W.make("normal", "float32", 200003, seed=10)
    t = to_device(x)
    assert bs.sort_(t, descending=True, mode=mode) is t
    assert_bit_exact(t.cpu().numpy(), O.bsort(x.copy(), descending=True), mode)
    with pytest.raises(ValueError):
        bs.sort_(t, mode="sideways")


def test_python_sort_segmented():
    import torch
    import paper_2603_08929_gb300 as bs
    sizes = np.array([3, 0, 5000, 1, 70000], dtype=np.int64)
    x = W.make("uniform", "int64", int(sizes.sum()), seed=11)
    off = np.concatenate([[0], np.cumsum(sizes)])
    t = to_device(x)
    bs.sort_segmented_(t, torch.from_numpy(off).cuda())
    got = t.cpu().numpy()
    for a, b in zip(off[:-1], off[1:]):
        assert_bit_exact(got[a:b], O.bsort(x[a:b].copy()), "segment [%d, %d)" % (a, b))
