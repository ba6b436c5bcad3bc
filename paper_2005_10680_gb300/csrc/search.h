// Host-side search for the first index at which a monotone predicate holds.
#pragma once

// Smallest k in [0, n) with pred(k) true, for a predicate that is false up to some
// index and true from there on; n when it is true nowhere. The search probes the
// hint (e.g. the previous selection) first, widens the bracket from there by
// doubling steps, then bisects inside it, so it returns the same index from any
// hint in [0, n).
//   eval(k, &pred, &value) -> status (0 = OK); the value at the returned index is
//   written to *at (left unchanged when the answer is n); *evals counts the calls.
template <class Eval>
int hinted_first_true(int n, int hint, Eval&& eval, int* answer, double* at, int* evals) {
    int lo = 0, hi = n;   // the answer lies in [lo, hi]; pred(hi) holds unless hi == n
    double vhi = 0.0, v = 0.0;
    bool p = false;
    int count = 0;
    int st = 0;
    if (hint < 0) hint = 0;
    if (hint > n - 1) hint = n - 1;
    if (n > 0) {
        st = eval(hint, &p, &v);
        ++count;
        if (st == 0 && p) {
            hi = hint;
            vhi = v;
            for (int step = 1; hi > lo && st == 0; step *= 2) {
                const int x = hi - step > lo ? hi - step : lo;
                st = eval(x, &p, &v);
                ++count;
                if (st != 0) break;
                if (p) {
                    hi = x;
                    vhi = v;
                } else {
                    lo = x + 1;
                    break;
                }
            }
        } else if (st == 0) {
            lo = hint + 1;
            for (int step = 1; lo < hi && st == 0; step *= 2) {
                const int x = lo + step - 1 < hi - 1 ? lo + step - 1 : hi - 1;
                st = eval(x, &p, &v);
                ++count;
                if (st != 0) break;
                if (p) {
                    hi = x;
                    vhi = v;
                    break;
                }
                lo = x + 1;
            }
        }
        while (lo < hi && st == 0) {
            const int mid = (lo + hi) / 2;
            st = eval(mid, &p, &v);
            ++count;
            if (st != 0) break;
            if (p) {
                hi = mid;
                vhi = v;
            } else {
                lo = mid + 1;
            }
        }
    }
    if (evals) *evals = count;
    if (st != 0) return st;
    *answer = hi;
    if (hi < n) *at = vhi;
    return 0;
}
