"""The read-bandwidth probe behind the memory roofline (needs a GB300): it
runs through the C ABI, a buffer inside the L2 reads faster than one four
times the L2's size, both rates are within physical bounds, and bad buffers
and sizes are refused before any launch."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_12786_gb300 import _build, vsr
    _build.build()
    return vsr


def _rate(V, buf, reps, trials=5):
    V.vsr_read_probe(buf, reps)
    best = 0.0
    for _ in range(trials):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        V.vsr_read_probe(buf, reps)
        b.record()
        torch.cuda.synchronize()
        best = max(best, buf.numel() * reps / (a.elapsed_time(b) / 1e3) / 1e9)
    return best


def test_l2_resident_reads_beat_hbm_reads(V):
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    small = torch.ones(l2 // 2 // 16 * 16, dtype=torch.uint8, device="cuda")
    large = torch.ones(4 * l2 // 16 * 16, dtype=torch.uint8, device="cuda")
    r_l2 = _rate(V, small, 20)
    r_hbm = _rate(V, large, 2)
    assert 1000.0 < r_hbm < 10000.0, r_hbm
    assert r_l2 > r_hbm, (r_l2, r_hbm)
    assert r_l2 < 100000.0, r_l2


def test_refusals(V):
    buf = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    with pytest.raises(V.VsrError, match="aligned"):
        V.vsr_read_probe(buf[1:17])
    with pytest.raises(V.VsrError, match="multiple of 16"):
        V.vsr_read_probe(buf[:24])
    with pytest.raises(V.VsrError, match="reps"):
        V.vsr_read_probe(buf, 0)
    with pytest.raises(V.VsrError, match="device memory|CUDA pointer"):
        V.vsr_read_probe(torch.zeros(64, dtype=torch.uint8))
    torch.cuda.synchronize()


def test_l1_probe_reads_faster_than_l2(V):
    """Every block re-reads a 32 KB buffer through L1: the launch reads more
    bytes per second than the L2-resident probe, within a physical bound."""
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    small = torch.ones(32 * 1024, dtype=torch.uint8, device="cuda")
    V.vsr_read_probe_l1(small, 64)
    best = 0.0
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        nbytes = V.vsr_read_probe_l1(small, 64)
        b.record()
        torch.cuda.synchronize()
        best = max(best, nbytes / (a.elapsed_time(b) / 1e3) / 1e9)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert nbytes % (32 * 1024 * 64) == 0 and nbytes // (32 * 1024 * 64) >= sms
    r_l2 = _rate(V, torch.ones(l2 // 2 // 16 * 16, dtype=torch.uint8, device="cuda"), 20)
    assert best > r_l2, (best, r_l2)
    assert best < 500000.0, best  # 152 SMs x 2 GHz x 1 KB/clk would be 311 TB/s


def test_l1_probe_refusals(V):
    buf = torch.zeros(1 << 17, dtype=torch.uint8, device="cuda")
    with pytest.raises(V.VsrError, match="65536"):
        V.vsr_read_probe_l1(buf)
    with pytest.raises(V.VsrError, match="reps"):
        V.vsr_read_probe_l1(buf[:4096], 0)
