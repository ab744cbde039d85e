"""The CPU oracle against its pins (worked examples of the paper, brute force,
ground truth of the generator, invariants, Graham's LPT bound)."""
import pytest

import oracle
from tests import _pins


@pytest.mark.parametrize("pin", _pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(oracle.default())


def test_pack2_hand_examples():
    """The 2-bit output layout on contigs packed by hand (the worked
    concatenation example of Sec. 4.4 and the reverse complement of Sec. 2)."""
    rows = _pins.golden("pack2_example.txt")
    for (k1, contig), (k2, *hexes) in zip(rows[0::2], rows[1::2]):
        assert k1 == "contig" and k2 == "bytes"
        assert oracle.pack2(contig.encode()).tobytes() == bytes(int(h, 16) for h in hexes)


def test_pack2_against_read_packing():
    """pack2 agrees with the generator's independent per-base packing of reads
    (the input layout) on random streams of every length mod 4."""
    import random
    import gen
    rnd = random.Random(5)
    for n in list(range(0, 12)) + [63, 64, 65, 1000]:
        s = "".join(rnd.choice("ACGT") for _ in range(n))
        want = gen.pack_reads([s])[2] if n else gen.pack_reads([s])[2][:0]
        assert oracle.pack2(s.encode()).tobytes() == want[: (n + 3) // 4].tobytes()
    with pytest.raises(ValueError):
        oracle.pack2(b"ACGN")
