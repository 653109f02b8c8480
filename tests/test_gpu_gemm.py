"""BF16 tensor-core GEMMs (tcgen05) against an FP64 matmul of the same BF16-rounded operands:
ragged row counts, two-source K, bias and relu, BF16 and FP32 outputs, accumulation, and the
row-reduction form A^T B used for weight gradients, and the time-out status of the bounded waits.
FP32 accumulation of K <= 256 products:
relative error <= 1e-5 before the output is rounded (BF16 output: half an ulp, 2^-9)."""
import numpy as np
import pytest

import sph_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_08919_gb300 import binding, build

    build.build()
    return binding, torch


def _bf16(torch, shape, seed, scale=1.0):
    v = (si.uniform53(seed, int(np.prod(shape))).reshape(shape) - 0.5) * 2 * scale
    return torch.tensor(v, dtype=torch.float32).to(torch.bfloat16)


# 200,003 rows: 1,563 row tiles, several for every persistent CTA, and a ragged last tile
@pytest.mark.parametrize("rows,K1,K2,N", [(1, 16, 0, 16), (128, 16, 16, 128), (300, 128, 32, 128),
                                          (1000, 32, 0, 32), (127, 128, 32, 160), (4099, 128, 0, 16),
                                          (200003, 128, 32, 128)])
def test_gemm_nt(env, rows, K1, K2, N):
    B, torch = env
    A1 = _bf16(torch, (rows, K1), 1)
    A2 = _bf16(torch, (rows, K2), 2) if K2 else None
    W = _bf16(torch, (N, K1 + K2), 3, 0.3)
    bias = torch.tensor(si.uniform53(4, N) - 0.5, dtype=torch.float32)
    A = torch.cat([A1, A2], 1) if K2 else A1
    ref = A.double() @ W.double().T + bias.double()
    d = {k: v.cuda() if v is not None else None for k, v in (("A1", A1), ("A2", A2), ("W", W), ("b", bias))}
    C = torch.zeros(rows, N, dtype=torch.float32, device="cuda")
    B.ann_bf16_gemm(d["A1"], d["W"], C, A2=d["A2"], bias=d["b"])
    err = (C.double().cpu() - ref).abs().max().item()
    assert err <= 1e-5 * ref.abs().max().item() + 1e-6, err
    Cb = torch.zeros(rows, N, dtype=torch.bfloat16, device="cuda")
    B.ann_bf16_gemm(d["A1"], d["W"], Cb, A2=d["A2"], bias=d["b"], relu=True)
    refr = ref.clamp(min=0.0)
    assert ((Cb.double().cpu() - refr).abs() <= 2.0 ** -8 * refr.abs() + 1e-6).all()
    C2 = C.clone()
    B.ann_bf16_gemm(d["A1"], d["W"], C2, A2=d["A2"], accumulate=True)
    assert (C2.double().cpu() - (C.double().cpu() + ref - bias.double())).abs().max().item() <= \
        2e-5 * ref.abs().max().item() + 1e-6


@pytest.mark.parametrize("rows,K,N", [(5, 16, 16), (128, 128, 32), (1000, 160, 128), (4099, 32, 16),
                                      (200003, 160, 128)])
def test_gemm_tn(env, rows, K, N):
    B, torch = env
    A = _bf16(torch, (rows, K), 11)
    G = _bf16(torch, (rows, N), 12)
    ref = A.double().T @ G.double()
    C = torch.full((K, N), 0.25, dtype=torch.float32, device="cuda")
    B.ann_bf16_gemm_tn(A.cuda(), G.cuda(), C)
    err = (C.double().cpu() - 0.25 - ref).abs().max().item()
    assert err <= 1e-5 * ref.abs().max().item() + 1e-5, err


def test_gemm_rejects_bad_shapes(env):
    B, torch = env
    A = torch.zeros(10, 24, dtype=torch.bfloat16, device="cuda")
    W = torch.zeros(16, 24, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(10, 16, dtype=torch.float32, device="cuda")
    with pytest.raises(B.AnnError):
        B.ann_bf16_gemm(A, W, C)   # K = 24 is not a multiple of 16


def test_an_expired_wait_is_a_status_not_a_hang(env):
    """The bounded mbarrier wait the tensor-core kernels use: waiting on a barrier nothing
    completes gives up after its poll limit and the host reads ANN_ERR_TIMEOUT; the device then
    runs a GEMM correctly."""
    B, torch = env
    assert B.ann_check_bounded_wait(4096) == -12
    assert B.ann_check_bounded_wait(1) == -12
    A = _bf16(torch, (300, 32), 21)
    W = _bf16(torch, (16, 32), 22)
    C = torch.zeros(300, 16, dtype=torch.float32, device="cuda")
    B.ann_bf16_gemm(A.cuda(), W.cuda(), C)
    ref = A.double() @ W.double().T
    assert (C.double().cpu() - ref).abs().max().item() <= 1e-5 * ref.abs().max().item() + 1e-6
