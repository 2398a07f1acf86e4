"""The allocation-free key switch (arx_keyswitch_noalloc) for callers that cannot
allocate device memory during a call (an HBM-budgeted server, a framework whose
allocator owns all device memory, a loop where cudaMalloc/cudaFree would
synchronise the device).

It must reproduce the gate path exactly: the LWE_N samples it is given are the
blind-rotation outputs of a batch of gates (computed here by the oracle, which the
GPU's blind rotation matches bit for bit), so its output must equal what
arx_bootstrap_gates_ex returns for the same gates -- tolerance 0, on two calls in
a row through the same shared scratch array.  This file is collected last so that
a run stopping at the first failure has already run every other test; it also
passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2306_11006_gb300 import arx
from paper_2306_11006_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_keyswitch_noalloc_matches_gate_path(O, keys630, torch_cuda):
    torch = torch_cuda
    n = keys630.n
    keyset = arx.load_keys(keys630.bsk, keys630.ksk, n)
    try:
        count = 24
        types = I.random_gate_types(900, count)
        ca = keys630.encrypt(O, I, I.random_bits(901, count), 902)
        cb = keys630.encrypt(O, I, I.random_bits(903, count), 904)
        # existing entry point: the full gate (blind rotation + key switch)
        want = np.zeros_like(ca)
        arx.bootstrap_gates_ex(types, ca, cb, None, want, keyset=keyset)
        # the same gates' blind-rotation outputs, as LWE_N samples [count][N+1]
        samples = np.stack([keys630.ctx.bootstrap_to_N(O.gate_linear(n, int(t), ca[g], cb[g]))
                            for g, t in enumerate(types)])
        d_samples = torch.from_numpy(samples.view(np.int32)).cuda()
        for call in range(2):
            d_out = torch.full((count, n + 1), -1, dtype=torch.int32, device="cuda")
            arx.keyswitch_noalloc(d_samples, d_out, keyset=keyset)
            got = d_out.cpu().numpy().view(np.uint32)
            assert np.array_equal(got, want), f"call {call}"
        # a different batch size through the same array, then the first one again
        d_out = torch.zeros((5, n + 1), dtype=torch.int32, device="cuda")
        arx.keyswitch_noalloc(d_samples[:5], d_out, count=5, keyset=keyset)
        assert np.array_equal(d_out.cpu().numpy().view(np.uint32), want[:5])
        # sizes beyond the fixed scratch are rejected, not truncated
        big = torch.zeros((arx.KS_NOALLOC_MAX + 1, arx.N + 1), dtype=torch.int32, device="cuda")
        big_out = torch.zeros((arx.KS_NOALLOC_MAX + 1, n + 1), dtype=torch.int32, device="cuda")
        with pytest.raises(arx.ArxError) as e:
            arx.keyswitch_noalloc(big, big_out, keyset=keyset)
        assert e.value.code == -1
    finally:
        arx.unload_keys(keyset)
