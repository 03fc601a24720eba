"""The sharded volume's exchange step over NCCL on the GPU (one rank): shard.volume runs the
rank-range split, reads this rank's partial sums and all-reduces them as device tensors through
an NCCL process group, which is the path each rank of a multi-GPU run takes.  The result must
be the oracle's exact volume."""

import json
import os
import socket

import pytest

import paper_1501_02237_gb300 as bd
from workloads import config_system

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_volumes.json")))["configs"]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("name", ["single_n24_k8", "small_n10_k4"])
def test_nccl_exchange_world_one(name):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.distributed as dist

    from paper_1501_02237_gb300 import shard

    torch.cuda.set_device(0)
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    store = dist.TCPStore("127.0.0.1", _free_port(), 1, True)
    dist.init_process_group("nccl", store=store, rank=0, world_size=1)
    try:
        assert dist.get_backend() == "nccl"
        P = bd.reduce(config_system(name).A)["points"]
        plan = bd.Plan(P)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            got = shard.volume(plan, seed=5, stream=stream)
        plan.close()
        assert got["nvol"] == GOLDEN[name]["nvol"]
        assert got["ties"] == 0 and got["cells"] > 0
        # the partial-sum exchange itself, on device tensors, with a value beyond 64 bits
        big = dict(nvol=(1 << 100) + 12345, cells=7, singular=3, ties=0)
        out = shard.combine(big)
        assert out["nvol"] == big["nvol"] and out["cells"] == 7 and out["singular"] == 3
    finally:
        dist.destroy_process_group()
