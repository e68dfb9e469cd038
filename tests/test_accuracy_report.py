"""The oracle's accuracy report runs on a small sample: every K-Best result stays at or above
the exact GED (checked inside the report), and the rates it prints are proportions."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import accuracy_report  # noqa: E402


def test_accuracy_report_small_sample(capsys):
    rows = accuracy_report.main(["--pairs-tiny", "24", "--pairs-molecule", "8", "--k-big", "300",
                                 "--ks", "1,16,64", "--threads", "2"])
    out = capsys.readouterr().out
    assert "| K | order | final step |" in out and "d(G,G) = 0" in out
    # K = 1, 64: both orders, variant A; K = 16 (the batch's own K): both orders, A and B
    assert len(rows) == 2 + 4 + 2
    for K, order, variant, exact, rel, worst in rows:
        assert 0.0 <= exact <= 1.0 and rel >= 0.0 and worst >= 0
        assert (exact == 1.0) == (worst == 0)
