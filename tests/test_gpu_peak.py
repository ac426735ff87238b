"""The measured-rate probes behind the rooflines (tcgen05 FP16 MMAs on CTA
pairs and single CTAs, MUFU ex2): they run, end cleanly and give rates in the
range a GB300 can reach (nominal dense FP16 2.25 PFLOP/s; ex2 at 16 to 32
results per clock per SM)."""
import pytest

import paper_2004_13653_gb300 as kde

pytestmark = pytest.mark.gpu


def test_peak_rates_are_plausible():
    r = kde.peak_rates()
    assert 800.0 < r["mma_f16_pair_tflops"] < 2600.0
    assert 400.0 < r["mma_f16_cta_tflops"] < 2600.0
    # 152 SMs x 16..32 per clock x 1.0..2.1 GHz
    assert 1.5 < r["ex2_tera_per_s"] < 25.0


def test_peak_rates_rejects_null():
    lib = kde.load()
    assert lib.kde_diag_peak_rates(None, None) == kde.KDE_EINVAL
