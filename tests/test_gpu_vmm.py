"""The memMap comparison array: a reserved range of device addresses grown
by mapping physical memory behind it keeps its address and its contents (no
copy), never shrinks, and refuses to grow past the reservation."""

import pytest
import torch

from paper_2209_00103_gb300 import gga

pytestmark = pytest.mark.gpu


def test_vmm_grows_in_place():
    v = gga.GGAVMM(1 << 30)
    inf = v.info()
    assert inf["mapped_bytes"] == 0 and inf["granularity"] > 0
    v.grow(10 << 20)
    n1 = (10 << 20) // 4
    a = v.tensor(n1)
    a.copy_(torch.arange(n1, dtype=torch.int32, device="cuda"))
    addr = v.info()["address"]
    v.grow(100 << 20)
    inf = v.info()
    assert inf["address"] == addr and inf["mapped_bytes"] >= 100 << 20
    assert inf["mapped_bytes"] % inf["granularity"] == 0
    b = v.tensor((100 << 20) // 4)
    assert torch.equal(b[:n1], torch.arange(n1, dtype=torch.int32, device="cuda"))
    b[n1:] = 7
    assert int(b[-1]) == 7 and int(b[n1 - 1]) == n1 - 1
    v.grow(5 << 20)                                           # never shrinks
    assert v.info()["mapped_bytes"] == inf["mapped_bytes"]
    with pytest.raises(gga.GGAError) as e:
        v.grow(2 << 30)
    assert e.value.code == gga.GGA_ERR_TOO_LARGE
    del a, b
    torch.cuda.synchronize()
    v.close()
