"""GPU data reductions of tests 35 and 100 (Sec. 4.2) against the oracle.

Counts are integers, so the GPU histograms and tables must equal the
oracle's exactly, per sequence, including gaps that cross the kernel's
16 384-value work units and sequences of every length.
"""
import numpy as np
import pytest

import oracle
from paper_1501_07701_gb300 import mtgp, quality, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
CHUNK = 1 << 14


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_07701_gb300 import build
    build.build()
    mtgp.load_library()


def _mtgp_outputs(counts, seed=0):
    """u32 outputs of len(counts) streams, back to back, on the device."""
    gp = mtgp.mtgp_params_generate(workloads.MEXP_MAIN, workloads.PARAM_SEED)
    st = mtgp.mtgp_init_statuses(gp, np.arange(seed, seed + len(counts), dtype=np.uint32))
    counts = np.asarray(counts, np.uint64)
    out = torch.empty(max(int(counts.sum()), 1), dtype=torch.int32, device="cuda")
    mtgp.mtgp_generate_u32(st, np.arange(len(counts)), counts, out)
    torch.cuda.synchronize()
    return out, counts


def _split(host, counts):
    offs = np.concatenate([[0], np.cumsum(counts.astype(np.int64))])
    return [host[offs[i]:offs[i + 1]] for i in range(len(counts))]


COUNTS = [3 * CHUNK + 17, 1, 0, 100, 2 * CHUNK, CHUNK - 1, 250000, 31, 32, 33]


@pytest.mark.parametrize("r,b,t", [(25, 5, 128), (0, 1, 16), (20, 10, 1023), (31, 1, 8), (25, 7, 300)])
def test_gap_histogram_matches_oracle(r, b, t):
    out, counts = _mtgp_outputs(COUNTS)
    hist = mtgp.mtgp_gap_histogram(out, counts, r=r, b=b, t=t)
    host = out.cpu().numpy().view(np.uint32)
    for i, seq in enumerate(_split(host, counts)):
        np.testing.assert_array_equal(hist[i], oracle.gap_histogram(seq, r=r, b=b, t=t),
                                      err_msg="sequence %d" % i)


def test_gap_histogram_visits_at_work_unit_edges():
    """Visits placed at and around the 16 384-value work-unit boundaries, a
    work unit without any visit, and a long first gap."""
    n = 5 * CHUNK + 9
    x = np.full(n, 0xFFFFFFFF, np.uint32)
    for p in [70000, CHUNK * 2 - 1, CHUNK * 2, CHUNK * 2 + 1, CHUNK * 4 + 5, n - 1]:
        x[p] = 0
    seqs = [x, x[:CHUNK * 2], np.zeros(40, np.uint32), x[CHUNK - 3:]]
    counts = np.array([s.size for s in seqs], np.uint64)
    dev = torch.from_numpy(np.concatenate(seqs).view(np.int32)).cuda()
    hist = mtgp.mtgp_gap_histogram(dev, counts, t=1023)
    for i, s in enumerate(seqs):
        np.testing.assert_array_equal(hist[i], oracle.gap_histogram(s, t=1023), err_msg="sequence %d" % i)
    assert hist[0].sum() == 6 and hist[0][70000 if 70000 < 1023 else 1023] >= 1


@pytest.mark.parametrize("r,s,L,bounds", [
    (25, 5, 1200, quality.default_hamming_bounds(1200, 4)),
    (25, 5, 1200, [600]),
    (0, 8, 64, list(range(18, 48, 2))),          # 16 classes
    (16, 16, 32, [14, 16, 18]),
    (28, 4, 400, []),                            # one class: the pair count
])
def test_hamming_pairs_match_oracle(r, s, L, bounds):
    counts = [3 * CHUNK + 17, 0, 2 * L // s * 3 - 1, 2 * L // s, 250000, 5, 0, 100000]
    out, counts = _mtgp_outputs(counts, seed=40)
    tab = mtgp.mtgp_hamming_pairs(out, counts, r=r, s=s, L=L, bounds=bounds)
    host = out.cpu().numpy().view(np.uint32)
    for i, seq in enumerate(_split(host, counts)):
        np.testing.assert_array_equal(tab[i], oracle.hamming_pairs(seq, r=r, s=s, L=L, bounds=bounds),
                                      err_msg="sequence %d" % i)


def test_statistics_of_mtgp_streams_pass():
    """Sanity: the pooled gap and Hamming statistics of a few seed-generated
    MTGP-11213 streams are not disastrous (p > 1e-6)."""
    pytest.importorskip("scipy")
    out, counts = _mtgp_outputs([1 << 22] * 4, seed=77)
    hist = mtgp.mtgp_gap_histogram(out, counts, t=128).sum(axis=0)
    bounds = quality.default_hamming_bounds(1200, 4)
    tab = mtgp.mtgp_hamming_pairs(out, counts, bounds=bounds).sum(axis=0)
    assert quality.gap_test(hist, b=5)["p_value"] > 1e-6
    assert quality.hamming_test(tab, L=1200, bounds=bounds)["p_value"] > 1e-6


def test_quality_argument_errors():
    out, counts = _mtgp_outputs([1000])
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_gap_histogram(out, counts, t=1024)
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_gap_histogram(out, counts, r=30, b=3)
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_hamming_pairs(out, counts, L=1201)
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_hamming_pairs(out, counts, bounds=list(range(16)))
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_hamming_pairs(out, counts, bounds=[610, 600])
