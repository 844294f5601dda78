"""GPU: the differentiable forms.  Sort-by-key and row permutation of float
payloads, checked by FP64 finite differences (gradcheck) at B=2, n=64 and
bit-exact against torch's stable sort + gather / scatter at B=64, n=65536 with
keys uniform on [0, 2^20) and N(0,1) upstream gradients."""
import numpy as np
import pytest

import synth
from helpers import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ag():
    import paper_1507_01391_b300 as m
    m.lib()
    from paper_1507_01391_b300 import autograd
    return autograd


def _bits(t):
    import torch
    return t.detach().contiguous().view(torch.int32 if t.dtype == torch.float32 else torch.int64)


def test_sort_by_key_gradcheck_fp64(ag):
    import torch
    B, n = 2, 64
    keys = dev(synth.uniform_keys(B * n, seed=1, bits=20).reshape(B, n))
    v = torch.from_numpy(synth.rng(2).standard_normal((B, n))).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: ag.sort_by_key(keys, x, 20)[1], (v,), eps=1e-6, atol=1e-9)


def test_permute_rows_gradcheck_fp64(ag):
    import torch
    B, n = 2, 64
    pi = dev(np.concatenate([synth.random_perm(n, seed=b) for b in range(B)]).reshape(B, n))
    v = torch.from_numpy(synth.rng(3).standard_normal((B, n))).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: ag.permute_rows(x, pi), (v,), eps=1e-6, atol=1e-9)


def test_sort_by_key_matches_torch_bit_exact(ag):
    import torch
    B, n = 64, 65536
    keys_np = synth.uniform_keys(B * n, seed=0x3A, bits=20).reshape(B, n)
    keys = dev(keys_np)
    v = torch.from_numpy(synth.normal_f32((B, n), seed=0x3B)).cuda().requires_grad_(True)
    g = torch.from_numpy(synth.normal_f32((B, n), seed=0x3C)).cuda()
    ko, y = ag.sort_by_key(keys, v, 20)
    y.backward(g)
    # torch reference: stable sort of the keys as int64, gather, pure-scatter backward
    k64 = torch.from_numpy(keys_np.astype(np.int64)).cuda()
    srt = torch.sort(k64, dim=1, stable=True)
    y_ref = torch.gather(v.detach(), 1, srt.indices)
    grad_ref = torch.zeros_like(v).scatter(1, srt.indices, g)
    assert torch.equal(ko.long() & 0xFFFFFFFF, srt.values)
    assert torch.equal(_bits(y), _bits(y_ref))
    assert torch.equal(_bits(v.grad), _bits(grad_ref))
    # torch's own autograd through gather accumulates into zeros: equal on N(0,1)
    v2 = v.detach().clone().requires_grad_(True)
    torch.gather(v2, 1, srt.indices).backward(g)
    assert torch.equal(_bits(v.grad), _bits(v2.grad))


def test_permute_rows_matches_torch_bit_exact(ag):
    import torch
    B, n = 64, 65536
    pi_np = np.concatenate([synth.random_perm(n, seed=100 + b) for b in range(B)]).reshape(B, n)
    pi = dev(pi_np)
    v = torch.from_numpy(synth.normal_f32((B, n), seed=0x3D)).cuda().requires_grad_(True)
    g = torch.from_numpy(synth.normal_f32((B, n), seed=0x3E)).cuda()
    y = ag.permute_rows(v, pi)
    y.backward(g)
    idx = torch.from_numpy(pi_np.astype(np.int64)).cuda()
    y_ref = torch.zeros_like(v).scatter(1, idx, v.detach())
    grad_ref = torch.gather(g, 1, idx)
    assert torch.equal(_bits(y), _bits(y_ref))
    assert torch.equal(_bits(v.grad), _bits(grad_ref))
