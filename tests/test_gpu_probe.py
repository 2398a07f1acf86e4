"""Integer-pipe probe (arx_probe_alu): the measured side of the ALU roofline."""
import pytest

from paper_2306_11006_gb300 import arx


@pytest.mark.gpu
def test_probe_rates_are_physical():
    r = arx.probe_alu()
    assert set(r) == set(arx.PROBE_NAMES)
    # an SM has 128 lanes: no 32-bit operation completes faster than that per clock
    assert all(0 < v <= 128 for v in r.values()), r
    # a butterfly costs several IMAD-class operations, more for the 64-bit prime
    assert r["shoup_bfly_q27"] < r["imad"]
    assert r["goldilocks_bfly"] < r["shoup_bfly_q27"]


@pytest.mark.gpu
def test_probe_rejects_bad_arguments():
    with pytest.raises(arx.ArxError):
        arx._check(arx.lib().arx_probe_alu(None, 7))
