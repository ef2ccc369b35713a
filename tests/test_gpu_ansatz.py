"""GPU parity of the ansatz (Sec. 3.1, mask of Sec. 3.3): log psi forward
and its reverse mode through the C ABI against the FP64 oracle, FP64 and
FP32 paths, including chunked batches and out-of-sector inputs.

Tolerances: FP64 path 1e-10 relative (different summation order only);
FP32 path 2e-4 absolute on log|psi| and phase (single rounding over ~10^2
accumulated terms per output); gradients relative to the largest entry of
each tensor: 1e-9 (FP64), 2e-3 (FP32), and for the BF16 reverse mode: every
GEMM of the reverse mode rounds both operands to BF16 (relative error 2^-9
each), and a weight gradient of layer l is a product chain through the
4 - l layers above it, two rounded operands per GEMM and three GEMMs per
layer on the path, so about 2 x 3 x 4 x 2^-9 = 0.047 of the tensor's scale in
the worst (first) layer: 4e-2 for NNQS_BF16X3, whose forward keeps about 16
operand bits.  NNQS_MIXED also rounds the forward's operands to BF16, and
the reverse mode reuses those activations: a second chain of the same
length, 2 x 0.047 = 0.094, so 1e-1 (measured: BF16X3 up to 8e-3, MIXED up
to 5.7e-2)."""
import numpy as np
import pytest
import torch

from oracle import ansatz as OA
from paper_2306_16705_gb300 import binding as B
from paper_2306_16705_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    B.lib()


def make(n_qubits, na, nb, d, L, H, seed, hidden=512, std=0.3):
    params = I.ansatz_params(n_qubits, d, L, seed, std=std, bias_std=0.1, phase_std=0.15)
    if hidden != 512:
        params = {k: v for k, v in params.items()}
        rng = np.random.default_rng(seed + 1)
        params["phase.w1"] = rng.normal(0, 0.15, (hidden, n_qubits)).astype(np.float32)
        params["phase.b1"] = rng.normal(0, 0.1, hidden).astype(np.float32)
        params["phase.w2"] = rng.normal(0, 0.15, (hidden, hidden)).astype(np.float32)
        params["phase.b2"] = rng.normal(0, 0.1, hidden).astype(np.float32)
        params["phase.w3"] = rng.normal(0, 0.15, (1, hidden)).astype(np.float32)
    m = B.Model(n_qubits, na, nb, d, L, H, hidden)
    return m, params, m.pack(params)


CASES = [  # (name, n_qubits, n_alpha, n_beta, d, L, heads, n_samples)
    ("n12", 12, 3, 3, 32, 2, 4, 400),
    ("n40", 40, 10, 10, 64, 4, 8, 300),
    ("w2", 70, 5, 6, 16, 2, 2, 100),
    ("dh16", 24, 4, 5, 64, 1, 4, 200),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [B.FP64, B.FP32])
def test_logpsi_matches_oracle(case, prec):
    name, N, na, nb, d, L, H, ns = case
    m, params, flat = make(N, na, nb, d, L, H, seed=11)
    x = I.random_sector_samples(N // 2, na, nb, ns, seed=3)
    got = B.logpsi(m, flat, B.to_device_bits(x), prec).cpu().numpy()
    la, ph = OA.forward(params, I.unpack_bits(x, N), na, nb, H)
    if prec == B.FP64:
        assert np.abs(got[:, 0] - la).max() <= 1e-10 * max(1.0, np.abs(la).max())
        assert np.abs(got[:, 1] - ph).max() <= 1e-10 * max(1.0, np.abs(ph).max())
    else:
        assert np.abs(got[:, 0] - la).max() <= 2e-4 * max(1.0, np.abs(la).max())
        assert np.abs(got[:, 1] - ph).max() <= 2e-4 * max(1.0, np.abs(ph).max())


def test_logpsi_normalised_on_gpu():
    """sum over the whole sector of |psi|^2 = exp(2 log|psi|) is 1."""
    m, params, flat = make(12, 3, 3, 32, 2, 4, seed=2)
    S = I.sector_states(6, 3, 3)
    lp = B.logpsi(m, flat, B.to_device_bits(S), B.FP64).cpu().numpy()
    assert abs(np.exp(2 * lp[:, 0]).sum() - 1.0) < 1e-12


def test_logpsi_chunked_batch():
    """More samples than one activation chunk: results are independent of the
    chunking (rows repeat; log psi needs no uniqueness)."""
    m, params, flat = make(12, 3, 3, 32, 2, 4, seed=5)
    S = I.sector_states(6, 3, 3)
    x = np.concatenate([S] * 90)  # 36000 rows > one chunk of 32768
    got = B.logpsi(m, flat, B.to_device_bits(x), B.FP64).cpu().numpy()
    ref = B.logpsi(m, flat, B.to_device_bits(S), B.FP64).cpu().numpy()
    assert np.array_equal(got, np.concatenate([ref] * 90))


def test_out_of_sector_reports_status():
    m, params, flat = make(12, 3, 3, 32, 2, 4, seed=5)
    x = I.sector_states(6, 3, 3)[:20].copy()
    x[4, 0] ^= np.uint64(1)
    with pytest.raises(B.NNQSError) as e:
        B.logpsi(m, flat, B.to_device_bits(x), B.FP64)
    assert e.value.status == B.E_SECTOR
    out = B.logpsi(m, flat, B.to_device_bits(x), B.FP64, check=False).cpu().numpy()
    assert out[4, 0] == -np.inf and np.all(np.isfinite(np.delete(out[:, 0], 4)))


GRAD_TOL = {B.FP64: 1e-9, B.FP32: 2e-3, B.MIXED: 1e-1, B.BF16X3: 4e-2}


@pytest.mark.parametrize("case", CASES[:3], ids=[c[0] for c in CASES[:3]])
@pytest.mark.parametrize("prec", [B.FP64, B.FP32, B.MIXED, B.BF16X3])
def test_backward_matches_oracle(case, prec):
    name, N, na, nb, d, L, H, ns = case
    ns = min(ns, 160)
    m, params, flat = make(N, na, nb, d, L, H, seed=13, hidden=96 if N > 40 else 512)
    x = I.random_sector_samples(N // 2, na, nb, ns, seed=4)
    rng = np.random.default_rng(0)
    seed = np.stack([rng.normal(size=ns), rng.normal(size=ns)], 1)
    g = B.logpsi_backward(m, flat, B.to_device_bits(x), torch.from_numpy(seed).cuda(), prec)
    G = m.unpack(g, params)
    _, _, cache = OA.forward(params, I.unpack_bits(x, N), na, nb, H, want_cache=True)
    R = OA.backward(cache, seed[:, 0], seed[:, 1])
    tol = GRAD_TOL[prec]
    worst = 0.0
    for k in params:
        ref = R[k]
        err = np.abs(G[k] - ref).max()
        worst = max(worst, err / max(1e-3, np.abs(ref).max()))
        assert err <= tol * max(1e-3, np.abs(ref).max()), (k, err, np.abs(ref).max())
    print(f"backward {name} prec={prec}: largest error / tensor scale = {worst:.3e}")


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_logpsi_mixed_tensor_cores(case):
    """NNQS_MIXED: linear layers on tcgen05 with BF16 operands and FP32
    accumulation.  BF16 keeps 8 significant bits, so log psi (a sum of T
    log-probabilities) is checked to 2e-2 of its scale against the FP64
    oracle, and must be far closer to it than a wrong kernel would be."""
    name, N, na, nb, d, L, H, ns = case
    m, params, flat = make(N, na, nb, d, L, H, seed=11)
    x = I.random_sector_samples(N // 2, na, nb, ns, seed=3)
    got = B.logpsi(m, flat, B.to_device_bits(x), B.MIXED).cpu().numpy()
    la, ph = OA.forward(params, I.unpack_bits(x, N), na, nb, H)
    assert np.abs(got[:, 0] - la).max() <= 2e-2 * max(1.0, np.abs(la).max())
    assert np.abs(got[:, 1] - ph).max() <= 2e-2 * max(1.0, np.abs(ph).max())
    # the error is at BF16 level, not at the level of an unrelated answer
    assert np.corrcoef(got[:, 0], la)[0, 1] > 0.999


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_logpsi_bf16x3_split_operands(case):
    """NNQS_BF16X3: the forward layers split X and W into high and low BF16
    parts and add three tensor-core products, so the operands keep about 16
    bits.  log psi is checked to 1e-3 of its scale against the FP64 oracle,
    and its error must be at least 20 times below that of single BF16
    operands on the same inputs."""
    name, N, na, nb, d, L, H, ns = case
    m, params, flat = make(N, na, nb, d, L, H, seed=11)
    x = I.random_sector_samples(N // 2, na, nb, ns, seed=3)
    xd = B.to_device_bits(x)
    got = B.logpsi(m, flat, xd, B.BF16X3).cpu().numpy()
    one = B.logpsi(m, flat, xd, B.MIXED).cpu().numpy()
    la, ph = OA.forward(params, I.unpack_bits(x, N), na, nb, H)
    ref = np.stack([la, ph], 1)
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(got - ref).max() <= 1e-3 * scale
    assert np.abs(got - ref).max() * 20 <= np.abs(one - ref).max()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_logpsi_fp8_tensor_cores(case):
    """NNQS_FP8: the forward layers on tcgen05 with E4M3 operands (weights
    scaled per row by a power of two).  E4M3 keeps 3 explicit mantissa bits
    against BF16's 7, a unit roundoff 16 times larger, so the NNQS_MIXED
    bound scales to 16 x 2e-2 = 0.32 of the log psi scale; the result must
    also follow the oracle (correlation > 0.95), which a wrong operand layout,
    scale or byte order would not."""
    name, N, na, nb, d, L, H, ns = case
    m, params, flat = make(N, na, nb, d, L, H, seed=11)
    x = I.random_sector_samples(N // 2, na, nb, ns, seed=3)
    got = B.logpsi(m, flat, B.to_device_bits(x), B.FP8).cpu().numpy()
    la, ph = OA.forward(params, I.unpack_bits(x, N), na, nb, H)
    err = max(np.abs(got[:, 0] - la).max(), np.abs(got[:, 1] - ph).max())
    scale = max(1.0, np.abs(la).max(), np.abs(ph).max())
    print(f"fp8 {name}: largest log psi error {err:.3e} of scale {scale:.2f}")
    assert err <= 0.32 * scale
    assert np.corrcoef(got[:, 0], la)[0, 1] > 0.95
    assert np.corrcoef(got[:, 1], ph)[0, 1] > 0.95


def test_backward_mixed_close_to_fp64():
    N, na, nb, d, L, H = 40, 10, 10, 64, 4, 8
    m, params, flat = make(N, na, nb, d, L, H, seed=13)
    x = B.to_device_bits(I.random_sector_samples(N // 2, na, nb, 200, seed=4))
    rng = np.random.default_rng(0)
    seed = torch.from_numpy(np.stack([rng.normal(size=200), rng.normal(size=200)], 1)).cuda()
    g64 = B.logpsi_backward(m, flat, x, seed, B.FP64).cpu().numpy()
    gmx = B.logpsi_backward(m, flat, x, seed, B.MIXED).cpu().numpy()
    assert np.linalg.norm(gmx - g64) <= 5e-2 * np.linalg.norm(g64)
    gx3 = B.logpsi_backward(m, flat, x, seed, B.BF16X3).cpu().numpy()
    assert np.linalg.norm(gx3 - g64) <= 5e-2 * np.linalg.norm(g64)


@pytest.mark.parametrize("prec", [B.FP64, B.FP32])
def test_backward_head_groups_match_oracle(prec):
    """120 qubits (60 tokens), d = 128, 8 heads: one sample's attention state
    is larger than a CTA's shared memory, so the attention reverse mode splits
    the heads over 2 (FP32) or 4 (FP64) CTAs per sample.  Gradients against
    the oracle's reverse mode with the tolerances above."""
    N, na, nb, d, L, H, ns = 120, 20, 20, 128, 1, 8, 12
    m, params, flat = make(N, na, nb, d, L, H, seed=17, hidden=64, std=0.1)
    x = I.random_sector_samples(N // 2, na, nb, ns, seed=5)
    rng = np.random.default_rng(2)
    seed = np.stack([rng.normal(size=ns), rng.normal(size=ns)], 1)
    g = B.logpsi_backward(m, flat, B.to_device_bits(x), torch.from_numpy(seed).cuda(), prec)
    G = m.unpack(g, params)
    _, _, cache = OA.forward(params, I.unpack_bits(x, N), na, nb, H, want_cache=True)
    R = OA.backward(cache, seed[:, 0], seed[:, 1])
    for k in params:
        err = np.abs(G[k] - R[k]).max()
        assert err <= GRAD_TOL[prec] * max(1e-3, np.abs(R[k]).max()), (k, err, np.abs(R[k]).max())


FUSED_CASES = [  # (name, n_qubits, n_alpha, n_beta, L, heads, n_samples): d = 64, FFN 256
    ("n40_ragged", 40, 10, 10, 4, 8, 1001),   # 6 samples of 20 tokens per 128-row tile, ragged last tile
    ("w2_t38", 76, 15, 15, 2, 8, 334),        # two words, 3 samples of 38 tokens per tile
    ("dh16_t12", 24, 4, 5, 1, 4, 500),        # head dimension 16, 10 samples per tile
    ("t64", 128, 30, 29, 1, 8, 40),           # 64 tokens: 2 samples per tile, two-word keys up to bit 127
]


@pytest.mark.parametrize("case", FUSED_CASES, ids=[c[0] for c in FUSED_CASES])
@pytest.mark.parametrize("prec", [B.MIXED, B.BF16X3])
def test_logpsi_fused_forward_matches_oracle(case, prec):
    """The fused forward (every decoder layer of a 128-row tile of token rows
    on chip, k_fwd_fused) that nnqs_logpsi and exact mode use for d = 64 in
    BF16 and split BF16: against the FP64 oracle with the bounds above
    (MIXED 2e-2, BF16X3 1e-3 of the log psi scale), over ragged tiles, two-word
    keys, head dimension 16 and T = 64."""
    name, N, na, nb, L, H, ns = case
    m, params, flat = make(N, na, nb, 64, L, H, seed=23, std=0.2)
    x = I.random_sector_samples(N // 2, na, nb, ns, seed=7)
    got = B.logpsi(m, flat, B.to_device_bits(x), prec).cpu().numpy()
    la, ph = OA.forward(params, I.unpack_bits(x, N), na, nb, H)
    ref = np.stack([la, ph], 1)
    scale = max(1.0, np.abs(ref).max())
    tol = 2e-2 if prec == B.MIXED else 1e-3
    err = np.abs(got - ref).max()
    print(f"fused {name} prec={prec}: largest log psi error {err:.3e} of scale {scale:.2f}")
    assert err <= tol * scale


def test_logpsi_fused_forward_two_chunks():
    """More samples than one chunk of 32,768: the fused path per chunk gives
    the same values as the samples evaluated alone (rows repeat)."""
    m, params, flat = make(40, 10, 10, 64, 2, 8, seed=24, std=0.2)
    S = I.random_sector_samples(20, 10, 10, 1000, seed=8)
    x = np.concatenate([S] * 34)  # 34,000 rows
    got = B.logpsi(m, flat, B.to_device_bits(x), B.BF16X3).cpu().numpy()
    one = B.logpsi(m, flat, B.to_device_bits(S), B.BF16X3).cpu().numpy()
    assert np.array_equal(got, np.concatenate([one] * 34))


@pytest.mark.parametrize("case", FUSED_CASES, ids=[c[0] for c in FUSED_CASES])
@pytest.mark.parametrize("prec", [B.MIXED, B.BF16X3])
def test_backward_fused_matches_oracle(case, prec):
    """The fused reverse mode of the decoder layers (k_bwd_ffn: one 128-row
    tile's FFN half with its forward recomputed on chip, weight gradients in
    TMEM over the CTA's tiles) that the BF16 and split-BF16 reverse modes use
    for d = 64: every gradient tensor of the transformer against the oracle's
    reverse mode with the BF16 bounds above, over ragged tiles, two-word keys,
    head dimension 16 and T = 64.  (The phase MLP is not part of the fused
    kernel; its gradient is checked above, and with BF16 forward operands a
    ReLU' that flips at a pre-activation near zero makes it discontinuous.)"""
    name, N, na, nb, L, H, ns = case
    ns = min(ns, 600)
    m, params, flat = make(N, na, nb, 64, L, H, seed=29, hidden=96, std=0.2)
    x = I.random_sector_samples(N // 2, na, nb, ns, seed=9)
    rng = np.random.default_rng(3)
    seed = np.stack([rng.normal(size=ns), rng.normal(size=ns)], 1)
    g = B.logpsi_backward(m, flat, B.to_device_bits(x), torch.from_numpy(seed).cuda(), prec)
    G = m.unpack(g, params)
    _, _, cache = OA.forward(params, I.unpack_bits(x, N), na, nb, H, want_cache=True)
    R = OA.backward(cache, seed[:, 0], seed[:, 1])
    worst = 0.0
    for k in (k for k in params if not k.startswith("phase.")):
        err = np.abs(G[k] - R[k]).max()
        worst = max(worst, err / max(1e-3, np.abs(R[k]).max()))
        assert err <= GRAD_TOL[prec] * max(1e-3, np.abs(R[k]).max()), (k, err, np.abs(R[k]).max())
    print(f"fused backward {name} prec={prec}: largest error / tensor scale = {worst:.3e}")
