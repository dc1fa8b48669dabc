/*
 * A plain C99 program against the C ABI of include/trw.h, built with
 * gcc -std=c99 -pedantic -Werror and linked against libtrw.so: the header is
 * C, and a C caller gets the documented statuses.  It runs without a GPU: it
 * calls entry points whose argument checks come before any CUDA call, plus
 * one load of a valid graph, whose status it prints (TRW_OK on a machine with
 * a GPU, TRW_ERR_CUDA on one without).  It also checks that trw_last_error()
 * is per thread: two threads that fail in turn each read their own message.
 * Exit status = the number of failed checks.
 */
#define _POSIX_C_SOURCE 200112L
#include <pthread.h>
#include <stdio.h>
#include <string.h>

#include "trw.h"

static int fails = 0;

#define CHECK(cond)                                                 \
  do {                                                              \
    if (!(cond)) {                                                  \
      fprintf(stderr, "abi_consumer.c:%d: %s\n", __LINE__, #cond); \
      ++fails;                                                      \
    }                                                               \
  } while (0)

static int says(const char* needle) {
  const char* m = trw_last_error();
  return m != NULL && strstr(m, needle) != NULL;
}

/* The two-vertex graph 0 -> 1, 1 -> 0 with a bad vertex array. */
static void invalid_graphs(void) {
  const int32_t col[2] = {1, 0};
  const int64_t good[3] = {0, 1, 2};
  const int64_t down[3] = {0, 2, 1};
  const int64_t start[3] = {1, 1, 2};
  trw_graph* g = (trw_graph*)&fails; /* not NULL: a failed load must clear it */

  CHECK(trw_graph_load(2, 2, good, col, NULL, NULL, 0, NULL) == TRW_ERR_INVALID);
  CHECK(says("out is NULL"));
  CHECK(trw_graph_load(-1, 2, good, col, NULL, NULL, 0, &g) == TRW_ERR_INVALID);
  CHECK(g == NULL);
  CHECK(trw_graph_load(2, 2, NULL, col, NULL, NULL, 0, &g) == TRW_ERR_INVALID);
  CHECK(says("row_ptr is NULL"));
  CHECK(trw_graph_load(2, 2, good, NULL, NULL, NULL, 0, &g) == TRW_ERR_INVALID);
  CHECK(says("col is NULL"));
  CHECK(trw_graph_load(2, 2, start, col, NULL, NULL, 0, &g) == TRW_ERR_INVALID);
  CHECK(says("row_ptr[0]"));
  CHECK(trw_graph_load(2, 2, down, col, NULL, NULL, 0, &g) == TRW_ERR_INVALID);
  CHECK(says("decreases"));
  CHECK(trw_graph_load(2, 3, good, col, NULL, NULL, 0, &g) == TRW_ERR_INVALID);
  CHECK(says("!= ne"));
}

static void null_handles(void) {
  trw_params p;
  int32_t src = 0, path[4], len;
  trw_server* s = NULL;
  memset(&p, 0, sizeof p);
  p.walks_per_source = 1;
  CHECK(trw_prepare(NULL, TRW_PREP_ALIAS) == TRW_ERR_INVALID);
  CHECK(trw_walk(NULL, TRW_DEEPWALK, &p, &src, 1, 3, 1, path, &len) == TRW_ERR_INVALID);
  CHECK(says("graph is NULL"));
  CHECK(trw_serve_create(NULL, NULL, &s) == TRW_ERR_INVALID);
  CHECK(s == NULL);
  trw_graph_free(NULL);
  trw_plan_destroy(NULL);
  trw_serve_destroy(NULL);
}

/* Thread-local messages: A fails, B fails differently, then A re-reads. */
static pthread_barrier_t bar;
static int thread_ok[2];

static void* fail_and_reread(void* arg) {
  const int me = *(const int*)arg;
  const int64_t rp[2] = {0, 0};
  trw_graph* g = NULL;
  if (me == 0) {
    trw_graph_load(1, 0, rp, NULL, NULL, NULL, 0, NULL); /* "out is NULL" */
    pthread_barrier_wait(&bar);
    pthread_barrier_wait(&bar); /* B has failed meanwhile */
    thread_ok[0] = says("out is NULL") && !says("row_ptr is NULL");
  } else {
    pthread_barrier_wait(&bar);
    trw_graph_load(1, 0, NULL, NULL, NULL, NULL, 0, &g); /* "row_ptr is NULL" */
    thread_ok[1] = says("row_ptr is NULL");
    pthread_barrier_wait(&bar);
  }
  return NULL;
}

static void thread_local_messages(void) {
  pthread_t t[2];
  int ids[2] = {0, 1};
  int i;
  CHECK(pthread_barrier_init(&bar, NULL, 2) == 0);
  for (i = 0; i < 2; ++i) CHECK(pthread_create(&t[i], NULL, fail_and_reread, &ids[i]) == 0);
  for (i = 0; i < 2; ++i) pthread_join(t[i], NULL);
  pthread_barrier_destroy(&bar);
  CHECK(thread_ok[0]);
  CHECK(thread_ok[1]);
}

int main(void) {
  const int64_t rp[4] = {0, 2, 4, 6};
  const int32_t col[6] = {1, 2, 0, 2, 0, 1}; /* a triangle */
  trw_graph* g = NULL;
  trw_status st;

  invalid_graphs();
  null_handles();
  thread_local_messages();

  st = trw_graph_load(3, 6, rp, col, NULL, NULL, 0, &g);
  CHECK((st == TRW_OK) == (g != NULL));
  if (st != TRW_OK) CHECK(trw_last_error() != NULL && trw_last_error()[0] != '\0');
  trw_graph_free(g);
  printf("load=%d fails=%d\n", (int)st, fails);
  return fails;
}
