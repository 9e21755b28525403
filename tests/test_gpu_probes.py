"""The measurement probes behind the bench's memory-side roofline (through the C ABI):
the read probe reads every byte of its buffer (its sum is checked), and the atomic
probe lands exactly n_updates / n_addr adds on every element, float and float4."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def abi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_01284_gb300 import abi
    abi.load()
    return abi


def test_read_probe_reads_everything(abi):
    g = torch.Generator(device="cuda").manual_seed(3)
    for n in (4, 1000, 1 << 20, (1 << 20) + 12):          # floats; ragged against the 4-load unroll
        buf = torch.randint(0, 4, (n,), device="cuda", generator=g).float()
        sink = torch.zeros(1, device="cuda")
        abi.pt_probe_read(buf, 3, sink)
        torch.cuda.synchronize()
        assert float(sink) == 3 * float(buf.sum()), n      # small integers: exact in FP32


@pytest.mark.parametrize("width", [1, 4])
@pytest.mark.parametrize("n_addr", [1, 32, 96, 1 << 20])
def test_atomic_probe_counts(abi, width, n_addr):
    per = 3
    dst = torch.zeros(n_addr * width, device="cuda")
    abi.pt_probe_atomic(dst, n_addr, per * n_addr, width)
    torch.cuda.synchronize()
    assert torch.all(dst == per)


def test_probe_argument_checks(abi):
    buf = torch.zeros(64, device="cuda")
    sink = torch.zeros(1, device="cuda")
    with pytest.raises(abi.PtError):
        abi.pt_probe_read(buf[1:], 1, sink)                  # not 16-byte aligned, size not a multiple of 16
    with pytest.raises(abi.PtError):
        abi.pt_probe_atomic(buf[1:], 4, 16, 4)               # float4 probe on an unaligned buffer
    with pytest.raises(abi.PtError):
        abi.pt_probe_atomic(buf, 4, 16, 3)                   # width must be 1 or 4
