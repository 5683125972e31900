"""The skewed full-size workload (500M records, Zipf 1.3 per byte with 10 %
duplicate keys, 4096 partitions) with the learned network requested, checked
through properties that hold at any size and together fix the result: the
output is sorted by key, equal keys keep input order (the record index rides
in the payload), and it is a permutation of the input byte for byte -- the
stable sort is the only sequence with all three.  The partitions stay within
1.1 x their mean (refined cuts), and the model choice is reported."""
import pytest
import torch

import paper_2305_05671_b300 as elsar
import recgen
from stable_check import check_stable_sort

pytestmark = pytest.mark.gpu

def test_zipf13_500M_network_requested():
    wl = recgen.ZIPF13_500M
    n, P = wl["n"], wl["P"]
    d_in = torch.empty(n * 100, dtype=torch.uint8, device="cuda")
    recgen.generate_gpu(d_in, n, wl["spec"])
    d_out = torch.empty_like(d_in)
    p = elsar.Params(num_partitions=P, model_kind=elsar.MODEL_MLP, seed=0x5EED)
    st = elsar.sort(d_in, d_out, n, p, stats=True)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    check_stable_sort(d_in, d_out, n)
    assert st["max_partition"] <= 1.1 * n / P
    assert st["model_used"] in (elsar.MODEL_RMI, elsar.MODEL_MLP)
    assert (st["model_used"] == elsar.MODEL_MLP) == (st["fallback_reason"] == 0)
    print("\nzipf1.3-500M:", st)
