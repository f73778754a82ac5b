"""Checkpoint and resume of the learned initialiser's trainer (host side, CPU tensors):
save() and load() restore the FP32 master weights, both Adam moments and the step
count bit for bit, rebuild the BF16 copy the layers read, and refuse a checkpoint
of another layer layout."""
import numpy as np
import pytest
import torch

from paper_2404_07780_b300 import cnn


def test_net_save_load_round_trip(tmp_path):
    net = cnn.Net(seed=3, device="cpu")
    g = torch.Generator().manual_seed(1)
    net.p.add_(torch.randn(net.n_params, generator=g) * 1e-3)   # as after some training
    net.m.copy_(torch.randn(net.n_params, generator=g))
    net.v.copy_(torch.rand(net.n_params, generator=g))
    net.step_count = 17
    path = tmp_path / "net.npz"
    net.save(path)
    back = cnn.Net.load(path, device="cpu")
    for name in ("p", "m", "v"):
        assert torch.equal(getattr(back, name), getattr(net, name)), name
    assert torch.equal(back.p_bf, net.p.to(torch.bfloat16))
    assert back.step_count == 17
    # a fresh network of the same seed differs: the restored weights are the checkpoint's
    assert not torch.equal(cnn.Net(seed=3, device="cpu").p, back.p)


def test_net_load_refuses_another_layout(tmp_path):
    net = cnn.Net(seed=0, device="cpu")
    path = tmp_path / "bad.npz"
    np.savez(path, p=net.p.numpy(), m=net.m.numpy(), v=net.v.numpy(), step=np.int64(0),
             offsets=net.offsets[:-1])
    with pytest.raises(ValueError, match="layer layout"):
        cnn.Net.load(path, device="cpu")
