"""The tcgen05 BF16 GEMM (C = A B^T, FP32 accumulation in tensor memory) against torch's matmul of
the same BF16 operands in FP32: the smallest tile first, then K loops longer than the copy ring,
256-wide tiles, split K and every epilogue."""
import numpy as np
import pytest

from paper_2411_05799_gb300 import npx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run(M, N, K, mode=npx.EPI_BIAS, splits=1, bias=True, want=("outf",), seed=0):
    g = torch.Generator(device="cpu").manual_seed(seed)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    b = (torch.randn(N, generator=g) if bias else torch.zeros(N)).float().cuda()
    zin = torch.randn(M, N, generator=g).to(torch.bfloat16).cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.full((M, N), float("nan"), dtype=torch.bfloat16, device="cuda")
    outT = torch.full((N, M), float("nan"), dtype=torch.bfloat16, device="cuda")
    outf = torch.full((splits, M, N), float("nan"), dtype=torch.float32, device="cuda")
    zsave = torch.full((M, N), float("nan"), dtype=torch.bfloat16, device="cuda")
    ep = npx.GemmEpilogue(mode=mode, bias=b.data_ptr() if bias and mode != npx.EPI_F32 else None,
                          out=out.data_ptr() if "out" in want else None, ldo=N,
                          outT=outT.data_ptr() if "outT" in want else None, ldt=M,
                          outf=outf.data_ptr() if "outf" in want else None, ldf=N,
                          split_stride=M * N,
                          zsave=zsave.data_ptr() if mode == npx.EPI_BIAS_GELU else None, ldz=N,
                          zin=zin.data_ptr(), ldzi=N)
    npx.gemm_bf16(A.data_ptr(), B.data_ptr(), M, N, K, ep, err.data_ptr(), splits=splits)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    acc = A.float() @ B.float().T
    return dict(A=A, B=B, b=b, zin=zin, acc=acc, out=out, outT=outT, outf=outf, zsave=zsave)


def _fp32_tol(K):
    """FP32 accumulation-order bound relative to the largest output: grows like sqrt(K)."""
    return 2e-7 * np.sqrt(K)


def _close(x, ref, rtol):
    """FP32 outputs: |x - ref| within rtol of the output's largest magnitude (the summation order
    of the FP32 accumulation differs from torch's); BF16 outputs: rtol per element."""
    x = x.double().cpu().numpy()
    ref = ref.double().cpu().numpy()
    if rtol < 1e-4:
        err = np.abs(x - ref).max() / np.abs(ref).max()
    else:
        err = (np.abs(x - ref) / (np.abs(ref) + 1e-2)).max()
    assert np.isfinite(x).all() and err <= rtol, err


def test_single_tile_single_k_block():
    r = _run(128, 128, 64)
    _close(r["outf"][0], r["acc"] + r["b"], _fp32_tol(64))


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 128, 320), (384, 512, 512), (512, 256, 1024)])
def test_tiles_and_long_k(M, N, K):
    r = _run(M, N, K, want=("outf", "out", "outT"))
    ref = r["acc"] + r["b"]
    _close(r["outf"][0], ref, _fp32_tol(K))
    _close(r["out"], ref, 8e-3)             # BF16 rounding of the output
    _close(r["outT"].T, ref, 8e-3)


def test_split_k_partials_sum_to_the_product():
    r = _run(256, 256, 2048, mode=npx.EPI_F32, splits=8, bias=False)
    _close(r["outf"].sum(0), r["acc"], _fp32_tol(2048))


# The epilogues take tanh from the special-function unit (relative error about 2^-11): a GELU
# value may move by 2^-11 |z| / 2 |t| and a GELU' value by 2^-11 |t| (1/2 + |z| k (1 + 3 c z^2) |t|),
# beside the FP32 rounding of the accumulation.
TANH_EPS = 2.0 ** -10.9
K_GELU, C_GELU = (2.0 / np.pi) ** 0.5, 0.044715


def test_gelu_and_dgelu_epilogues():
    """Bias + GELU and GELU' against torch's GELU in its tanh form on the same accumulators."""
    r = _run(256, 512, 320, mode=npx.EPI_BIAS_GELU, want=("outf", "out"))
    z = r["acc"] + r["b"]
    _close(r["zsave"], z, 8e-3)
    z64 = z.double().cpu().numpy()
    t = np.tanh(K_GELU * (z64 + C_GELU * z64 ** 3))
    bound = TANH_EPS * 0.5 * np.abs(z64) * np.abs(t) + _fp32_tol(320) * np.abs(z64).max()
    got = r["outf"][0].double().cpu().numpy()
    ref = torch.nn.functional.gelu(z.double(), approximate="tanh").cpu().numpy()
    assert (np.abs(got - ref) <= bound).all(), np.max(np.abs(got - ref) / bound)
    r = _run(256, 256, 256, mode=npx.EPI_DGELU, bias=False, want=("outf",))
    zin = r["zin"].double().cpu().numpy()
    acc = r["acc"].double().cpu().numpy()
    t = np.tanh(K_GELU * (zin + C_GELU * zin ** 3))
    du = K_GELU * (1.0 + 3.0 * C_GELU * zin * zin)
    dg = 0.5 * (1.0 + t) + 0.5 * zin * (1.0 - t * t) * du
    bound = (np.abs(acc) * TANH_EPS * np.abs(t) * (0.5 + np.abs(zin) * du * np.abs(t))
             + _fp32_tol(256) * np.abs(acc * dg).max())
    got = r["outf"][0].double().cpu().numpy()
    assert (np.abs(got - acc * dg) <= bound).all(), np.max(np.abs(got - acc * dg) / bound)


def test_rejects_bad_shapes():
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    A = torch.zeros(128, 64, dtype=torch.bfloat16, device="cuda")
    ep = npx.GemmEpilogue(mode=npx.EPI_BIAS, outf=A.data_ptr())
    with pytest.raises(npx.NpxError):
        npx.gemm_bf16(A.data_ptr(), A.data_ptr(), 100, 128, 64, ep, err.data_ptr())
    with pytest.raises(npx.NpxError):
        npx.gemm_bf16(A.data_ptr(), A.data_ptr(), 128, 128, 96, ep, err.data_ptr())
