"""The cluster chain's byte-counted exchanges (host arithmetic only): for every
grid size, node count and cluster size the chain can run with, the bytes each
CTA expects on its two mbarriers per time average equal the bytes the other
CTAs send it -- the partial sums of its own (branch, wavenumber) pairs from
every rank, and the whole state from the owners -- so no wait can run out in
a correct run.  The ownership arithmetic is the kernel's: C CTAs, own =
ceil(K1/C) wavenumbers each, CTA j owning [min(K1, j own), min(K1, (j+1) own));
rank j sends the sum for pair (b, k) to CTA k // own; owner thread (b, r)
sends its result to every CTA.  The counts the kernel arms its mbarriers with
come from the library itself (arp_chain_exchange_bytes runs the kernel's own
host-and-device function), for both precisions."""
import pytest

from _helpers import built_library


def _exchange(K1, C):
    own = -(-K1 // C)
    rng = [(min(K1, j * own), min(K1, j * own + own)) for j in range(C)]
    red_sent = [0] * C
    for _rank in range(C):
        for i in range(3 * K1):
            red_sent[(i % K1) // own] += 1
    ws_sent = [0] * C
    for o in range(C):
        k0, k1 = rng[o]
        for _pair in range(3 * (k1 - k0)):
            for c in range(C):
                ws_sent[c] += 1
    red_expected = [C * 3 * (k1 - k0) for k0, k1 in rng]
    ws_expected = [3 * K1] * C
    return red_sent, red_expected, ws_sent, ws_expected, rng


@pytest.mark.parametrize("N", [8, 16, 32, 64, 128, 256, 512, 1024, 2048])
@pytest.mark.parametrize("C", [8, 16])
def test_expected_bytes_equal_sent_bytes(N, C):
    K1 = (N - 1) // 3 + 1
    red_sent, red_expected, ws_sent, ws_expected, rng = _exchange(K1, C)
    assert red_sent == red_expected
    assert ws_sent == ws_expected
    # the owned ranges tile 0..K1-1 exactly once; a CTA owning nothing expects no partial sums
    owned = [k for k0, k1 in rng for k in range(k0, k1)]
    assert owned == list(range(K1))
    assert all(e == 0 for (k0, k1), e in zip(rng, red_expected) if k1 == k0)


@pytest.mark.parametrize("N,C", [(512, 16), (2048, 16), (64, 16)])
def test_byte_counts_fit_the_transaction_counter(N, C):
    # an mbarrier's pending transaction count holds at most 2^20 - 1 bytes; the
    # largest phase carries 16-byte FP64 complex values
    K1 = (N - 1) // 3 + 1
    _, red_expected, _, ws_expected, _ = _exchange(K1, C)
    assert max(red_expected) * 16 < (1 << 20) - 1
    assert max(ws_expected) * 16 < (1 << 20) - 1


@pytest.mark.parametrize("N", [8, 16, 64, 128, 512, 1024, 2048])
@pytest.mark.parametrize("C", [1, 4, 8, 16])
@pytest.mark.parametrize("precision,elem", [(0, 16), (1, 8)], ids=["fp64", "fp32"])
def test_kernel_byte_counts_equal_sent_bytes(N, C, precision, elem):
    # what the kernel expects (the library's arithmetic) against what the other
    # CTAs send (the model above), in bytes of the precision's complex values
    built_library()
    from paper_1303_6615_gb300 import binding as b
    K1 = (N - 1) // 3 + 1
    red_sent, _, ws_sent, _, _ = _exchange(K1, C)
    for rank in range(C):
        red, ws = b.arp_chain_exchange_bytes(N, C, rank, precision)
        assert red == red_sent[rank] * elem, (rank, red, red_sent[rank])
        assert ws == ws_sent[rank] * elem, (rank, ws, ws_sent[rank])


def test_kernel_byte_counts_reject_bad_arguments():
    built_library()
    from paper_1303_6615_gb300 import binding as b
    for args in ((500, 16, 0, 0), (512, 17, 0, 0), (512, 16, 16, 0), (512, 16, -1, 0), (512, 16, 0, 2)):
        with pytest.raises(b.ArpError) as ei:
            b.arp_chain_exchange_bytes(*args)
        assert ei.value.status == b.ARP_EINVAL
