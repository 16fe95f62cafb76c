"""Arrays past the 32-bit signed (and, for 1-byte keys, unsigned) index
range.  Key positions, bucket starts, chunk starts and counts are 64-bit
through the whole pipeline, so positions above 2^31 and element counts above
2^32 must land exactly like small ones.  Checked byte for byte against the
oracle's output where the host holds it beside the input (about 7x the keys'
bytes for 4-byte keys), else by the properties that pin a sort at any size:
non-decreasing under the oracle's order, the input's multiset, and sampled
positions holding the key of their rank."""
import pytest

import workloads as W
from gpu_util import check_by_properties, check_full_size

pytestmark = pytest.mark.gpu

N31 = (1 << 31) + 1234567  # 4-byte keys: 8.6 GB, every chunk past 2^31 has a position above INT32_MAX
N32 = (1 << 32) + 777      # 1-byte keys: more keys than a uint32 counts


def _host_bytes_free():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2603_08929_gb300 import build as b
    b.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("mode,desc", [("pingpong", False), ("inplace", True)])
def test_int32_past_2p31(mode, desc):
    import torch
    import paper_2603_08929_gb300 as bs
    x = W.make("uniform", "int32", N31, seed=31)
    t = torch.from_numpy(x).cuda()
    bs.sort_(t, descending=desc, mode=mode)
    got = t.cpu().numpy()
    del t
    torch.cuda.empty_cache()
    if _host_bytes_free() > 8 * x.nbytes:
        check_full_size(x, got, desc)
    else:
        check_by_properties(x, got, desc, samples=6, seed=1)


def test_uint8_past_2p32():
    import torch
    import paper_2603_08929_gb300 as bs
    x = W.make("uniform", "uint8", N32, seed=32)
    t = torch.from_numpy(x).cuda()
    bs.sort_(t)
    got = t.cpu().numpy()
    del t
    torch.cuda.empty_cache()
    check_full_size(x, got, False)
