"""Product shards of one trajectory simulated on the GPU one after another (the
work each rank of a sharded job does), joined on the host: the actions at their
times, the cost and lost totals and the final stock rows are the whole
trajectory's (the oracle's sequential path), and every shard's actions are its
own Picard fixed point."""
import numpy as np
import pytest

import oracle
from paper_2406_01939_b300 import shard, synth
from paper_2406_01939_b300.session import DeviceInstance
from paper_2406_01939_b300.synth import Policy

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 4, 7])
def test_product_shards_on_gpu_join_to_the_sequential_path(world):
    inst = synth.dual_large(3, T=1 << 18, K=3000, R=300)
    pol = Policy("dual")
    want = oracle.seq_sim(inst, pol)
    owner = shard.product_shards(inst.prod, inst.K, world)
    full = np.full(inst.T, -2, np.int8)
    cost = lost = 0
    for r in range(world):
        sub, times, mine = shard.shard_instance(inst, owner, r)
        got = DeviceInstance(sub).simulate(pol, "picard", num_chunks=256)
        full[times] = got["actions"].cpu().numpy()
        cost += got["total_cost"]
        lost += got["lost"]
        np.testing.assert_array_equal(got["final_stock"].cpu().numpy(), want["x_final"][mine])
    np.testing.assert_array_equal(full, want["actions"])
    assert cost == want["total_cost"] and lost == want["lost"]


def test_mlp_product_shards_on_gpu():
    inst = synth.make_instance(20000, 32, 60, 40, seed=5, stock="poisson", fill=0.8)
    pol = Policy("mlp", mlp=synth.make_mlp(32, 40, seed=5))
    want = oracle.seq_sim(inst, pol)
    owner = shard.product_shards(inst.prod, inst.K, 3)
    full = np.full(inst.T, -2, np.int8)
    for r in range(3):
        sub, times, _ = shard.shard_instance(inst, owner, r)
        full[times] = DeviceInstance(sub).simulate(pol, "picard", num_chunks=64)["actions"].cpu().numpy()
    np.testing.assert_array_equal(full, want["actions"])
