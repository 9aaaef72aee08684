"""GPU: the float32 FMA-throughput probe (tlrmvn_measure_fp32_peak) against the
device's nominal rate: SMs x 128 FP32 lanes x 2 flops x maximum SM clock.  The
probe runs eight independent FMA chains per thread at full occupancy, so it must
land between half of that rate and the rate itself (plus timing slack)."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_fp32_peak_is_near_the_nominal_rate():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    import paper_2003_11183_gb300 as tl
    props = torch.cuda.get_device_properties(0)
    try:
        import subprocess
        mhz = float(subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                                    "-i", "0"], capture_output=True, text=True, timeout=60).stdout.split()[0])
    except Exception:
        mhz = 2070.0
    nominal = props.multi_processor_count * 128 * 2 * mhz * 1e6 / 1e12
    got = max(tl.tlrmvn_measure_fp32_peak() for _ in range(3))
    assert 0.5 * nominal < got < 1.05 * nominal, (got, nominal)
